// Residual / energy sums that allocate nothing, for callers that cannot call
// cudaMalloc (see lbm_residual_noalloc in phonon_lbm.h).  The per-block
// partial sums live in a fixed file-scope device array instead of memory
// from the allocator.
#include <cmath>
#include <mutex>

#include "../../include/phonon_lbm.h"
#include "lbm_kernels.h"

namespace {

constexpr int NODES_PER_BLOCK = 4096;      // 256 threads x 16 nodes
constexpr int MAX_BLOCKS = 4096;           // -> at most 16,777,216 nodes
constexpr int MAX_DEVICES = 64;

// Partial sums of every block (5 doubles each), then the 5 final sums.
// 163,880 bytes, held by every device that loads the library until exit.
static __device__ __align__(256) double g_noalloc_scratch[MAX_BLOCKS * 5 + 5];

std::mutex g_mu;
double *g_scratch_ptr[MAX_DEVICES] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One block reduces its 4096-node slice into 5 partials (same sums as the
// context's residual pass): sum de, sum de^2, sum |q|^2, sum |(de,q) - prev|^2,
// count of non-finite nodes, with de = e - e_ref.
__global__ void __launch_bounds__(256)
slice_sums(const double *__restrict__ e, const double *__restrict__ qx,
           const double *__restrict__ qy, const double *__restrict__ pe,
           const double *__restrict__ pqx, const double *__restrict__ pqy, long long n,
           double e_ref, double *__restrict__ scratch) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * NODES_PER_BLOCK;
    const bool have_prev = pe != nullptr;
#pragma unroll 4
    for (int j = 0; j < NODES_PER_BLOCK / 256; ++j) {
        const long long i = base + j * 256 + threadIdx.x;
        if (i >= n) break;
        const double de = e[i] - e_ref, a = qx[i], b = qy[i];
        if (!(isfinite(de) && isfinite(a) && isfinite(b))) acc[4] += 1.0;
        acc[0] += de;
        acc[1] += de * de;
        acc[2] += a * a + b * b;
        if (have_prev) {
            const double u = de - (pe[i] - e_ref), v = a - pqx[i], w = b - pqy[i];
            acc[3] += u * u + v * v + w * w;
        }
    }
    __shared__ double sh[5][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double s = warp_sum(acc[q]);
        if (lane == 0) sh[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[threadIdx.x][w];
        scratch[blockIdx.x * 5 + threadIdx.x] = s;
    }
}

// Fixed-order sum of the block partials into scratch[MAX_BLOCKS*5 + q].
__global__ void __launch_bounds__(256) total_sums(double *__restrict__ scratch, int blocks) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < blocks; b += 256) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += scratch[b * 5 + q];
    }
    __shared__ double sh[5][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double s = warp_sum(acc[q]);
        if (lane == 0) sh[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[threadIdx.x][w];
        scratch[MAX_BLOCKS * 5 + threadIdx.x] = s;
    }
}

// Failures are reported through lbm_last_error(NULL); a CUDA failure is
// also cleared from the runtime's per-thread error record once reported.
lbm_status noalloc_fail(lbm_status s, const char *msg) {
    plbm::set_global_error(msg);
    if (s == LBM_ECUDA) (void)cudaGetLastError();
    return s;
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is not a device address).
lbm_status scratch_address(double **out) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return noalloc_fail(LBM_ECUDA, cudaGetErrorString(err));
    if (dev < 0 || dev >= MAX_DEVICES) return noalloc_fail(LBM_EUNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess || !p) return noalloc_fail(LBM_ECUDA, cudaGetErrorString(err));
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_residual_noalloc(const double *e, const double *qx, const double *qy,
                                const double *prev_e, const double *prev_qx,
                                const double *prev_qy, long long n_nodes, double e_ref,
                                long k_steps, void *stream, double *r, double *total_energy) {
    if (!e || !qx || !qy) return noalloc_fail(LBM_EINVAL, "e, qx and qy must be device arrays");
    const bool have_prev = prev_e || prev_qx || prev_qy;
    if (have_prev && !(prev_e && prev_qx && prev_qy))
        return noalloc_fail(LBM_EINVAL, "give all three previous fields or none");
    if (n_nodes < 1) return noalloc_fail(LBM_EINVAL, "n_nodes must be >= 1");
    static_assert((long long)MAX_BLOCKS * NODES_PER_BLOCK == LBM_NOALLOC_MAX_NODES,
                  "header limit and scratch size disagree");
    if (n_nodes > LBM_NOALLOC_MAX_NODES)
        return noalloc_fail(LBM_EINVAL,
                            "n_nodes exceeds the 16777216-node maximum of the "
                            "no-allocation residual (its fixed scratch holds 4096 "
                            "block partials of 4096 nodes); use lbm_residual");
    if (!std::isfinite(e_ref)) return noalloc_fail(LBM_EINVAL, "e_ref is not finite");
    double *scratch = nullptr;
    if (lbm_status s = scratch_address(&scratch)) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)((n_nodes + NODES_PER_BLOCK - 1) / NODES_PER_BLOCK);
    // every partial slot the sum reads is written first by its block, so
    // nothing left over from an earlier call is ever read
    slice_sums<<<blocks, 256, 0, st>>>(e, qx, qy, prev_e, prev_qx, prev_qy, n_nodes, e_ref,
                                       scratch);
    total_sums<<<1, 256, 0, st>>>(scratch, blocks);
    cudaError_t err = cudaGetLastError();
    double sums[5];
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(sums, scratch + MAX_BLOCKS * 5, sizeof(sums),
                              cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return noalloc_fail(LBM_ECUDA, cudaGetErrorString(err));
    const double n = (double)n_nodes;
    const double mean = sums[0] / n;
    const double var_e = std::fmax(sums[1] - n * mean * mean, 0.0);
    const double denom = std::sqrt(var_e + sums[2]);
    double res = INFINITY;
    if (have_prev && k_steps > 0) {
        const double num = std::sqrt(sums[3]);
        res = denom > 0.0 ? num / ((double)k_steps * denom) : (num == 0.0 ? 0.0 : INFINITY);
    }
    if (r) *r = res;
    if (total_energy) *total_energy = n * e_ref + sums[0];
    if (sums[4] > 0.0) return noalloc_fail(LBM_ENONFINITE, "fields hold NaN or Inf");
    return LBM_OK;
}

}  // extern "C"
