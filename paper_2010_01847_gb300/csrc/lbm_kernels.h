// Internal launch interface between the C-ABI layer and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace plbm {

enum { PREC_FP32 = 0, PREC_FP16 = 1, PREC_BF16 = 2, PREC_FP64 = 3 };
enum { KERNEL_AUTO = 0, KERNEL_SCALAR = 1, KERNEL_VECTOR = 2, KERNEL_STAGED = 3 };

// Sets the text lbm_last_error(NULL) returns.
void set_global_error(const char *msg);

// Elements per 16-byte vector for a storage kind.
int vector_width(int precision);

// One time step: src (post-collision, step n-1) -> dst (post-collision, step n).
template <typename T>
cudaError_t launch_step(int kernel, const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                        const Coef<typename Store<T>::C> &k, cudaStream_t stream);

// The bulk-copy staged variant (see staged.cu).  Returns
// cudaErrorNotSupported when the lattice does not meet its layout rules.
template <typename T>
cudaError_t launch_step_staged(const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                               const Coef<typename Store<T>::C> &k, cudaStream_t stream);
bool staged_supported(int precision, int nx, int ny);

// Read-out of the state at the current step.  `pulled` = the state is the
// pull of the post-collision planes in `src` (step >= 1); otherwise `src`
// holds the state itself (step 0).
struct Readout {
    int nx, ny, bc_x, bc_y;
    bool pulled;
    double e_ref;     // reference energy of the deviations
    double inv_scale; // 1 / storage scale
    double kappa;     // Eq. 54 factor
};

template <typename T>
cudaError_t launch_moments(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                           double *e, double *qx, double *qy, cudaStream_t stream);

template <typename T>
cudaError_t launch_populations(const T *src, const Readout &r,
                               const Coef<typename Store<T>::C> &k, double *f,
                               cudaStream_t stream);

// Residual pass: per node e, q of the state; accumulates in FP64
//   sums[0] = sum (e - e_ref), sums[1] = sum (e - e_ref)^2,
//   sums[2] = sum |q|^2, sums[3] = sum |(e,q) - prev|^2 (if have_prev),
//   sums[4] = count of non-finite e or q,
// and overwrites prev[3][n] with the current (e - e_ref, qx, qy).
// `partials` holds RESIDUAL_BLOCKS*5 doubles of scratch.
constexpr int RESIDUAL_BLOCKS = 1216;    // 8 blocks per SM on 152 SMs
template <typename T>
cudaError_t launch_residual(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                            double *prev, bool have_prev, double *partials, double *sums,
                            cudaStream_t stream);

// Initial state from device fields (Eq. 15): writes the state of step 0 into
// `pre` and its collision into `post`.  qx/qy may be null.
template <typename T>
cudaError_t launch_init(const double *e, const double *qx, const double *qy, int nx, int ny,
                        double e_ref, double scale, const Coef<typename Store<T>::C> &k, T *pre,
                        T *post, cudaStream_t stream);

// Largest |w e - w e_ref| + |5/3 a c.q| bound over nodes, for the 16-bit
// scale: writes max over nodes of (2/9)|e - e_ref| + (1/3)(|qx| + |qy|) into
// *out (device, must start at 0) as the bit pattern of a double.
cudaError_t launch_max_deviation(const double *e, const double *qx, const double *qy,
                                 long long n, double e_ref, unsigned long long *out,
                                 cudaStream_t stream);

}  // namespace plbm
