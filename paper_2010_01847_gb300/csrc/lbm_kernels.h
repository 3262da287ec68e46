// Internal launch interface between the C-ABI layer and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm_device.cuh"

namespace plbm {

// Names a host-side call on profiler timelines (NVTX range; costs nothing
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

enum { PREC_FP32 = 0, PREC_FP16 = 1, PREC_BF16 = 2, PREC_FP64 = 3 };
enum { KERNEL_AUTO = 0, KERNEL_SCALAR = 1, KERNEL_VECTOR = 2, KERNEL_STAGED = 3,
       KERNEL_RESIDENT = 4, KERNEL_WAVE = 5 };

// 16-bit storage keeps a plane of tile references after the 8 population
// planes (refs16.cuh): tiles of 8 nodes when nx is a multiple of 8, else of
// one node.  tile_shift_of: 3 or 0 for 16-bit storage, -1 for the others.
inline bool has_tile_refs(int precision) {
    return precision == PREC_FP16 || precision == PREC_BF16;
}
inline int tile_shift_of(int precision, int nx) {
    return !has_tile_refs(precision) ? -1 : (nx % 8 == 0 ? 3 : 0);
}
// Elements of the storage type in one state buffer of an nx x ny lattice.
inline long long state_elems(int precision, int nx, int ny) {
    const long long plane = (long long)nx * ny;
    const int sh = tile_shift_of(precision, nx);
    return 8 * plane + (sh < 0 ? 0 : 8 * (plane >> sh));
}
// The tile-reference fields of the coefficients (after the weights are set):
// the reference populations R_i = 4 w_i rho~ + 4 h_i c_i . j~ of a stored
// {rho, j} / 4, the tile-sum factors 1 / (4 nodes-per-tile) for rho and
// gamma / (4 nodes-per-tile) for the flux, gamma = 1 - omega lambda -
// sigma (1 - lambda) the factor the collision applies to m = sum c_i d_i
// (Eqs. 15, 16 and 54 summed against c_i).
template <typename C>
inline void set_tile_refs(Coef<C> &k, int precision, int nx, int ny, double tau, double tau_r) {
    k.tile_shift = tile_shift_of(precision, nx);
    if (k.tile_shift < 0) return;
    k.tiles_x = nx >> k.tile_shift;
    k.ref_off = 8LL * nx * ny;
    k.rw_axis = (C)4 * k.w_axis;
    k.rw_diag = (C)4 * k.w_diag;
    k.rh_axis = (C)4 * k.h_axis;
    k.rh_diag = (C)4 * k.h_diag;
    const double per_tile = 4.0 * (double)(1 << k.tile_shift);
    const double omega = 1.0 / tau;
    const bool resistive = tau_r < 1e300;
    const double lambda = resistive ? 1.0 / (2.0 * tau_r + 1.0) : 0.0;
    const double sigma = resistive ? (1.0 - 1.0 / (2.0 * tau)) / tau_r : 0.0;
    const double gamma = 1.0 - omega * lambda - sigma * (1.0 - lambda);
    k.ref_rho = (C)(1.0 / per_tile);
    k.ref_gamma = (C)(gamma / per_tile);
}

// Sets the text lbm_last_error(NULL) returns.
void set_global_error(const char *msg);

// Elements per 16-byte vector for a storage kind.
int vector_width(int precision);

// Launch shape of the staged kernel.
struct StagedPlan {
    int stages = 2;          // shared-memory ring depth
    int ctas_per_sm = 0;     // persistent CTAs per SM
    int grid = 0;            // SMs x ctas_per_sm
    int consumer_warps = 8;  // 4 or 8: tile width 32 x consumer_warps x V nodes
    int hint = 0;            // L2 evict-first policy on the bulk loads
};

// Computes a staged plan on the current device (sets the kernel's shared
// memory attribute; call outside stream capture).  stages <= 0 = default 2;
// ctas_per_sm <= 0 = as many as fit; consumer_warps <= 0 = 8.
cudaError_t staged_plan(int precision, int stages, int ctas_per_sm, int consumer_warps,
                        int l2_hint, StagedPlan *out);
int staged_tile_width(int precision, int consumer_warps);

// One time step: src (post-collision, step n-1) -> dst (post-collision,
// step n).  With rq non-null the launch also computes the residual sums of
// the state at step n (5 doubles per block into rq->partials; *blocks_out
// receives the block count).  `status` is a device word the staged kernel
// sets when a bounded wait gives up.
template <typename T>
cudaError_t launch_step(int kernel, const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                        const Coef<typename Store<T>::C> &k, int *status,
                        const ResidualReq<typename Store<T>::C> *rq, const StagedPlan &plan,
                        int *blocks_out, cudaStream_t stream);

// Plain steps of 16-bit storage on the vector layout (pipe16.cu): a
// persistent kernel; prepare_pipe16 sets it up on the current device
// (launch attributes, grid size; call outside stream capture), the launch
// returns cudaErrorNotReady without it.
cudaError_t prepare_pipe16(int precision);
template <typename T>
cudaError_t launch_step_pipe16(const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                               const Coef<float> &k, cudaStream_t stream);

// Largest number of blocks a step launch of this kernel can have (sizes the
// per-block residual partials).
long long step_blocks(int kernel, int precision, int nx, int ny, const StagedPlan &plan);

// The bulk-copy staged variant (see staged.cu); plain steps only (a step
// with the fused residual runs on the vector kernel).
template <typename T>
cudaError_t launch_step_staged(const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                               const Coef<typename Store<T>::C> &k, int *status,
                               const StagedPlan &plan, int *blocks_out, cudaStream_t stream);
bool staged_supported(int precision, int nx, int ny, int consumer_warps);

// Launch shape of the cluster-resident kernel (resident.cu): one cluster of
// `cluster` CTAs, CTA r owning slab r of w columns (part_x) or rows.
struct ResidentPlan {
    int cluster = 0;    // CTAs in the one cluster (0: no plan)
    int part_x = 0;     // 1: slabs of columns, 0: slabs of rows
    int w = 0;          // columns (rows) per slab
    int rows = 0;       // allocated rows of a slab plane (ghost rows included)
    int cols = 0;       // allocated columns (ghost columns included)
    int last_rank = 0;  // the last CTA with nodes
    int npt = 0;        // nodes per thread (1..4)
    int threads = 0;    // threads per CTA
    int smem = 0;       // dynamic shared memory per CTA (bytes)
};

// A plan for an FP32 lattice whose two post-collision buffers fit in the
// shared memory of one cluster (cluster_req > 0 asks for that many CTAs);
// cudaErrorNotSupported when none fits or none can be resident on this
// device.  Sets the kernel's launch attributes: call outside stream capture.
cudaError_t resident_plan(int precision, int nx, int ny, int cluster_req, ResidentPlan *out);

// `steps` (>= 1) time steps from the post-collision planes `src`: writes the
// post-collision planes of the last step to out_last and of the step before
// it to out_prev (src may be either; each CTA reads its own nodes before it
// writes them).  `status`: the device word a bounded wait that gives up sets
// (bit 2).
cudaError_t launch_resident(const float *src, float *out_last, float *out_prev, int nx, int ny,
                            int bc_x, int bc_y, const Coef<float> &k, long steps,
                            const ResidentPlan &p, int *status, cudaStream_t stream);

// The multi-step kernel (wave.cu): `steps` (WAVE_MIN_STEPS..WAVE_MAX_STEPS)
// time steps in one launch, src (post-collision, step n) -> dst
// (post-collision, step n + steps); the post-collision state of step
// n + steps - 1 is not kept.  Strips of 64 columns, segments of seg_rows rows
// (clipped to ny).  cudaErrorInvalidValue for lattices it does not take
// (wave_supported) or src == dst.
constexpr int WAVE_MIN_STEPS = 2;
constexpr int WAVE_MAX_STEPS = 8;
constexpr int WAVE16_MAX_STEPS = 4;     // 16-bit storage (wave16.cu)
bool wave_supported(int precision, int nx, int ny, int bc_x, int bc_y);
int wave_max_steps(int precision);
cudaError_t launch_step_wave(int steps, const float *src, float *dst, int nx, int ny, int bc_x,
                             int bc_y, const Coef<float> &k, int seg_rows, cudaStream_t stream);
// The same for FP16 / BF16 storage with tile references (nx % 8 == 0): level
// 0 decoded, levels in FP32, level `steps` stored against the reference of
// level steps - 1 (rounded once per launch).
cudaError_t launch_step_wave16(int precision, int steps, const void *src, void *dst, int nx,
                               int ny, int bc_x, int bc_y, const Coef<float> &k, int seg_rows,
                               cudaStream_t stream);
// Runs the staged kernel's bounded mbarrier wait against a barrier nothing
// completes (one CTA, ~2 s); the wait gives up and ORs 1 into *status.
cudaError_t launch_wait_probe(int *status, cudaStream_t stream);
// The same for the cluster-resident kernel's ghost wait (one-CTA cluster);
// ORs 2 into *status.
cudaError_t launch_resident_wait_probe(int *status, cudaStream_t stream);

// Blocks of the stand-alone residual pass (sizes its per-block partials).
long long readout_blocks(int precision, int nx, int ny, int bc_x, int bc_y);

// Fixed-order sum of per-block partials (5 doubles each) into sums[0..4].
// With `mid` (room for FINALIZE_MID x 5 doubles) and more than
// FINALIZE_SPLIT blocks it takes two launches: FINALIZE_MID blocks each sum
// a contiguous run of partials in order, then one block sums their results
// in order (still a fixed order: the result does not vary between runs).
// Returns the number of launches in *launches when non-null.
constexpr int FINALIZE_MID = 128;
constexpr int FINALIZE_SPLIT = 8192;
cudaError_t launch_finalize(const double *partials, int blocks, double *sums,
                            cudaStream_t stream, double *mid = nullptr, int *launches = nullptr);

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

// Stand-alone residual pass over the state at the current step: the same
// per-node sums as the fused step variant (residual_node in lbm_device.cuh),
// 5 partial sums per block into `partials` (RESIDUAL_BLOCKS blocks), then
// the fixed-order total into `sums`.
constexpr int RESIDUAL_BLOCKS = 1216;    // 8 blocks per SM on 152 SMs
template <typename T>
cudaError_t launch_residual(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                            typename Store<T>::C *prev, bool have_prev, double *partials,
                            double *sums, cudaStream_t stream, double *mid = nullptr);

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
