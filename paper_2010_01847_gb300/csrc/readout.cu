// Initialisation and read-out kernels: Eq. 15 initial state, moments
// (Eqs. 53-54), raw populations, and the FP64 residual / energy reduction.
// None of these is on the per-step path; they run once per read-out.
#include "lbm_kernels.h"

namespace plbm {

// Populations of the state at the current step for node (x, y), as the
// stream-collide kernel sees them before colliding.
template <typename T>
__device__ __forceinline__ void state_node(const T *__restrict__ src, const Readout &r,
                                           const Coef<typename Store<T>::C> &k, int x, int y,
                                           typename Store<T>::C (&d)[8]) {
    const long long plane = (long long)r.nx * r.ny;
    if (r.pulled) {
        pull_node<T>(src, plane, r.nx, r.ny, x, y, r.bc_x, r.bc_y, k, d);
    } else {
        const long long node = (long long)y * r.nx + x;
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = Store<T>::load(src[(long long)i * plane + node]);
    }
}

// e - e_ref, qx, qy of one node in FP64 (sums in FP64 of the stored values).
template <typename C>
__device__ __forceinline__ void node_moments_f64(const C (&d)[8], const Readout &r, double &de,
                                                 double &qx, double &qy) {
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (double)d[i];
    const double rho = ((v[0] + v[2]) + (v[1] + v[3])) + ((v[4] + v[6]) + (v[5] + v[7]));
    const double mx = (v[0] - v[2]) + (v[4] - v[6]) + (v[7] - v[5]);
    const double my = (v[1] - v[3]) + (v[4] - v[6]) + (v[5] - v[7]);
    de = rho * r.inv_scale;
    qx = r.kappa * mx * r.inv_scale;
    qy = r.kappa * my * r.inv_scale;
}

template <typename T>
__global__ void moments_kernel(const T *__restrict__ src, Readout r,
                               Coef<typename Store<T>::C> k, double *e, double *qx,
                               double *qy) {
    using C = typename Store<T>::C;
    const long long n = (long long)r.nx * r.ny;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = int(node / r.nx), x = int(node - (long long)y * r.nx);
        C d[8];
        state_node<T>(src, r, k, x, y, d);
        double de, a, b;
        node_moments_f64(d, r, de, a, b);
        if (e) e[node] = r.e_ref + de;
        if (qx) qx[node] = a;
        if (qy) qy[node] = b;
    }
}

// Weights of Eq. 17, for adding back the rest-state part of a deviation.
__device__ __forceinline__ double omega_of(int i) { return i < 4 ? 2.0 / 9.0 : 1.0 / 36.0; }

template <typename T>
__global__ void populations_kernel(const T *__restrict__ src, Readout r,
                                   Coef<typename Store<T>::C> k, double *f) {
    using C = typename Store<T>::C;
    const long long n = (long long)r.nx * r.ny;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = int(node / r.nx), x = int(node - (long long)y * r.nx);
        C d[8];
        state_node<T>(src, r, k, x, y, d);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            f[(long long)i * n + node] = (double)d[i] * r.inv_scale + omega_of(i) * r.e_ref;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
residual_kernel(const T *__restrict__ src, Readout r, Coef<typename Store<T>::C> k,
                typename Store<T>::C *__restrict__ prev, int have_prev,
                double *__restrict__ partials) {
    using C = typename Store<T>::C;
    const long long n = (long long)r.nx * r.ny;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = int(node / r.nx), x = int(node - (long long)y * r.nx);
        C d[8];
        state_node<T>(src, r, k, x, y, d);
        residual_node(d, k, (C)r.inv_scale, prev, n, node, have_prev != 0, acc);
    }
    block_sum5_store(acc, partials + (size_t)blockIdx.x * 5);
}

// Fixed-order sum of the per-block partials (deterministic result).
__global__ void __launch_bounds__(256) finalize_sums(const double *__restrict__ partials,
                                                     int blocks, double *__restrict__ sums) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += partials[b * 5 + q];
    }
    block_sum5_store(acc, sums);
}

template <typename T>
__global__ void init_kernel(const double *__restrict__ e, const double *__restrict__ qx,
                            const double *__restrict__ qy, int nx, int ny, double e_ref,
                            double scale, Coef<typename Store<T>::C> k, T *__restrict__ pre,
                            T *__restrict__ post) {
    using C = typename Store<T>::C;
    const long long n = (long long)nx * ny;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const double de = e[node] - e_ref;
        const double a = qx ? qx[node] : 0.0;
        const double b = qy ? qy[node] : 0.0;
        // Eq. 15 on deviations: w_i (e - e_ref) + (5/3) a_i c_i.q, times s;
        // (5/3) a_i = 1/3 (axis) or 1/12 (diagonal).
        const double dv[8] = {
            (2.0 / 9.0) * de + a / 3.0,          (2.0 / 9.0) * de + b / 3.0,
            (2.0 / 9.0) * de - a / 3.0,          (2.0 / 9.0) * de - b / 3.0,
            (1.0 / 36.0) * de + (a + b) / 12.0,  (1.0 / 36.0) * de + (b - a) / 12.0,
            (1.0 / 36.0) * de - (a + b) / 12.0,  (1.0 / 36.0) * de + (a - b) / 12.0};
        C d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const T s = Store<T>::put((C)(dv[i] * scale));
            pre[(long long)i * n + node] = s;
            d[i] = Store<T>::load(s);
        }
        collide(d, k);
#pragma unroll
        for (int i = 0; i < 8; ++i) post[(long long)i * n + node] = Store<T>::put(d[i]);
    }
}

__global__ void max_deviation_kernel(const double *__restrict__ e, const double *__restrict__ qx,
                                     const double *__restrict__ qy, long long n, double e_ref,
                                     unsigned long long *out) {
    double m = 0.0;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        double v = (2.0 / 9.0) * fabs(e[node] - e_ref);
        if (qx) v += fabs(qx[node]) / 3.0;
        if (qy) v += fabs(qy[node]) / 3.0;
        m = isfinite(v) ? fmax(m, v) : HUGE_VAL;   // non-finite input -> +inf
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

static unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    return (unsigned)(b > 0 ? b : 1);
}

template <typename T>
cudaError_t launch_moments(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                           double *e, double *qx, double *qy, cudaStream_t stream) {
    moments_kernel<T><<<grid_for((long long)r.nx * r.ny, 256), 256, 0, stream>>>(src, r, k, e,
                                                                               qx, qy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_populations(const T *src, const Readout &r,
                               const Coef<typename Store<T>::C> &k, double *f,
                               cudaStream_t stream) {
    populations_kernel<T><<<grid_for((long long)r.nx * r.ny, 256), 256, 0, stream>>>(src, r, k,
                                                                                   f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                            typename Store<T>::C *prev, bool have_prev, double *partials,
                            double *sums, cudaStream_t stream) {
    residual_kernel<T><<<RESIDUAL_BLOCKS, 256, 0, stream>>>(src, r, k, prev, have_prev ? 1 : 0,
                                                            partials);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_finalize(partials, RESIDUAL_BLOCKS, sums, stream);
}

cudaError_t launch_finalize(const double *partials, int blocks, double *sums,
                            cudaStream_t stream) {
    finalize_sums<<<1, 256, 0, stream>>>(partials, blocks, sums);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init(const double *e, const double *qx, const double *qy, int nx, int ny,
                        double e_ref, double scale, const Coef<typename Store<T>::C> &k, T *pre,
                        T *post, cudaStream_t stream) {
    init_kernel<T><<<grid_for((long long)nx * ny, 256), 256, 0, stream>>>(e, qx, qy, nx, ny,
                                                                        e_ref, scale, k, pre,
                                                                        post);
    return cudaGetLastError();
}

cudaError_t launch_max_deviation(const double *e, const double *qx, const double *qy,
                                 long long n, double e_ref, unsigned long long *out,
                                 cudaStream_t stream) {
    max_deviation_kernel<<<grid_for(n, 256), 256, 0, stream>>>(e, qx, qy, n, e_ref, out);
    return cudaGetLastError();
}

#define PLBM_INSTANTIATE(T)                                                                   \
    template cudaError_t launch_moments<T>(const T *, const Readout &,                        \
                                           const Coef<Store<T>::C> &, double *, double *,     \
                                           double *, cudaStream_t);                           \
    template cudaError_t launch_populations<T>(const T *, const Readout &,                    \
                                               const Coef<Store<T>::C> &, double *,           \
                                               cudaStream_t);                                 \
    template cudaError_t launch_residual<T>(const T *, const Readout &,                       \
                                            const Coef<Store<T>::C> &, Store<T>::C *, bool,   \
                                            double *, double *, cudaStream_t);                \
    template cudaError_t launch_init<T>(const double *, const double *, const double *, int,  \
                                        int, double, double, const Coef<Store<T>::C> &, T *,  \
                                        T *, cudaStream_t);

PLBM_INSTANTIATE(float)
PLBM_INSTANTIATE(double)
PLBM_INSTANTIATE(__half)
PLBM_INSTANTIATE(__nv_bfloat16)

}  // namespace plbm
