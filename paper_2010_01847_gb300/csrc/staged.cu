// Staged stream-collide kernel: the bulk-copy engine (TMA) moves row
// segments of all 8 planes into a ring of shared-memory stages while the
// consumer warps collide the previous stage.
//
// Tile = one row segment of W = 32 CW V nodes (CW consumer warps, V =
// 16 / sizeof(T)), i.e. 512 CW bytes per plane, plus one 16-byte halo vector
// on each side.  Plane i of
// output row y is pulled from row y - c_iy (Eq. 13, left-hand side), so the
// producer copies, for each plane, that source row's segment
// [x0 - V, x0 + W + V) (split at the x seam, where the halo wraps to the far
// end of the row).  Every copy starts on a 16-byte boundary and is a multiple
// of 16 bytes, as the bulk copy requires.
//
// Roles per CTA: warp CW lane 0 is the producer (waits until a stage is free,
// arms the stage's "full" mbarrier with the byte count, issues
// cp.async.bulk for the 8 plane segments); warps 0..CW-1 consume (wait "full",
// pull from shared memory, seam/wall rules, collide, store 16-byte vectors
// straight to global memory, release the stage on its "empty" mbarrier).
// CTAs are persistent: tile t goes to CTA t mod gridDim.
//
// Every wait is bounded (iteration and clock limits).  A wait that gives up
// sets bit 1 of *status and the role stops; the producer then waits (again
// bounded) until every copy it issued has landed before the CTA can exit.
#include <type_traits>

#include "lbm_kernels.h"
#include "mbarrier.cuh"

namespace plbm {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return smem_u32(p); }

// Bounded wait of this kernel (sets STATUS_STAGED when it gives up).
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity, int *status) {
    return mbar_wait<false>(bar, parity, status, STATUS_STAGED);
}

// Global -> shared bulk copy completing on an mbarrier (the TMA engine).
// With `hinted`, the copy carries an L2 evict-first policy (the data is read
// exactly once per step).
__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *bar, bool hinted, uint64_t policy) {
    if (hinted)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
            "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst_smem)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(smem_addr(dst_smem)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar))
            : "memory");
}

__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void st_stream(void *p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

template <typename T> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int V = 4;
    __device__ static void unpack(uint4 r, float (&o)[4]) {
        o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
        o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
    }
    __device__ static uint4 pack(const float (&o)[4]) {
        return make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                          __float_as_uint(o[3]));
    }
};
template <> struct Vec16<double> {
    static constexpr int V = 2;
    __device__ static void unpack(uint4 r, double (&o)[2]) {
        o[0] = __hiloint2double((int)r.y, (int)r.x);
        o[1] = __hiloint2double((int)r.w, (int)r.z);
    }
    __device__ static uint4 pack(const double (&o)[2]) {
        return make_uint4((unsigned)__double2loint(o[0]), (unsigned)__double2hiint(o[0]),
                          (unsigned)__double2loint(o[1]), (unsigned)__double2hiint(o[1]));
    }
};

template <typename T, int CW> constexpr int tile_width() { return CW * 32 * Vec16<T>::V; }
template <typename T, int CW> constexpr int row_len() {
    return tile_width<T, CW>() + 2 * Vec16<T>::V;
}
template <typename T, int CW> constexpr int stage_bytes() {
    return 8 * row_len<T, CW>() * (int)sizeof(T);
}

template <typename T, int CW>
__global__ void __launch_bounds__((CW + 1) * 32, 1)
step_staged(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny, long long plane,
            int bc_x, int bc_y, int stages, int hinted, Coef<typename Store<T>::C> k,
            int *status) {
    using C = typename Store<T>::C;
    constexpr int V = Vec16<T>::V;
    constexpr int W = tile_width<T, CW>();
    constexpr int RL = row_len<T, CW>();
    constexpr int SB = stage_bytes<T, CW>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)stages * SB);
    uint64_t *empty = full + stages;

    const int tiles_per_row = nx / W;
    const long long n_tiles = (long long)tiles_per_row * ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (warp == CW) {
        // ---------------- producer ----------------
        if (lane == 0) {
            const uint64_t policy = hinted ? evict_first_policy() : 0ull;
            long long issued = 0;
            for (long long tile = blockIdx.x, kk = 0; tile < n_tiles;
                 tile += gridDim.x, ++kk) {
                const int s = (int)(kk % stages);
                const uint32_t ph = (uint32_t)((kk / stages) & 1);
                if (!stage_wait(&empty[s], ph ^ 1u, status)) break;
                const int y = (int)(tile / tiles_per_row);
                const int x0 = (int)(tile - (long long)y * tiles_per_row) * W;
                mbar_expect_tx(&full[s], (uint32_t)SB);
                T *stage = ring + (size_t)s * 8 * RL;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    int sy = y - cy_of(i);
                    sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                    const T *row = src + (long long)i * plane + (long long)sy * nx;
                    T *d = stage + i * RL;
                    if (x0 > 0 && x0 + W < nx) {
                        bulk_copy(d, row + x0 - V, RL * sizeof(T), &full[s], hinted, policy);
                    } else {
                        bulk_copy(d, row + (x0 == 0 ? nx - V : x0 - V), V * sizeof(T), &full[s],
                                  hinted, policy);
                        bulk_copy(d + V, row + x0, W * sizeof(T), &full[s], hinted, policy);
                        bulk_copy(d + V + W, row + (x0 + W == nx ? 0 : x0 + W), V * sizeof(T),
                                  &full[s], hinted, policy);
                    }
                }
                issued = kk + 1;
            }
            // every copy issued must land before the CTA may exit
            for (long long kk = issued > stages ? issued - stages : 0; kk < issued; ++kk)
                stage_wait(&full[kk % stages], (uint32_t)((kk / stages) & 1), status);
        }
    } else {
        // ---------------- consumers ----------------
        const int t = threadIdx.x;          // owns nodes x0 + t V .. + V - 1
        const bool walls = bc_y == BC_WALLS;
        for (long long tile = blockIdx.x, kk = 0; tile < n_tiles; tile += gridDim.x, ++kk) {
            const int s = (int)(kk % stages);
            const uint32_t ph = (uint32_t)((kk / stages) & 1);
            if (!stage_wait(&full[s], ph, status)) break;
            const int y = (int)(tile / tiles_per_row);
            const int x0 = (int)(tile - (long long)y * tiles_per_row) * W;
            const T *stage = ring + (size_t)s * 8 * RL;
            const bool bottom = walls && y == 0;
            const bool top = walls && y == ny - 1;
            const long long out = (long long)y * nx + x0 + t * V;
            {     // V nodes per consumer thread
                C d[8][V];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const T *r = stage + i * RL + V + t * V;
                    Vec16<T>::unpack(*reinterpret_cast<const uint4 *>(r), d[i]);
                    const int cx = cx_of(i);
                    if (cx > 0) {
                        C left = Store<T>::load(r[-1]);
                        if (bc_x == BC_GRADIENT && x0 == 0 && t == 0)
                            left += (i < 4) ? k.jump_axis : k.jump_diag;     // Eq. 59
#pragma unroll
                        for (int j = V - 1; j >= 1; --j) d[i][j] = d[i][j - 1];
                        d[i][0] = left;
                    } else if (cx < 0) {
                        C right = Store<T>::load(r[V]);
                        if (bc_x == BC_GRADIENT && x0 + W == nx && t == CW * 32 - 1)
                            right -= (i < 4) ? k.jump_axis : k.jump_diag;    // Eq. 60
#pragma unroll
                        for (int j = 0; j < V - 1; ++j) d[i][j] = d[i][j + 1];
                        d[i][V - 1] = right;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);     // this warp is done with the stage
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    C n[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) n[i] = d[i][j];
                    if (bottom) wall_bottom(n, k);
                    if (top) wall_top(n, k);
                    collide(n, k);
#pragma unroll
                    for (int i = 0; i < 8; ++i) d[i][j] = n[i];
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    st_stream(dst + (long long)i * plane + out, Vec16<T>::pack(d[i]));
            }
        }
    }
}

constexpr int MAX_STAGES = 6;

template <typename T, int CW>
constexpr size_t smem_bytes(int stages) {
    return (size_t)stages * stage_bytes<T, CW>() + 2 * (size_t)stages * sizeof(uint64_t);
}

template <typename T> constexpr int prec_of() {
    return sizeof(T) == 4 ? PREC_FP32 : PREC_FP64;
}

template <typename T, int CW> constexpr auto kernel_of() { return step_staged<T, CW>; }

struct DeviceInfo {
    int sms = 0;
    bool prepared[4][2] = {};   // per storage kind, per consumer-warp variant
};
DeviceInfo g_info[64];

// Once per device, storage kind and variant: allow the kernel's largest ring.
template <typename T, int CW>
cudaError_t prepare(int dev) {
    DeviceInfo &info = g_info[dev];
    if (!info.sms) {
        cudaError_t e = cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int vi = CW == 8 ? 0 : 1;
    if (!info.prepared[prec_of<T>()][vi]) {
        int optin = 0;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        const int want = (int)smem_bytes<T, CW>(MAX_STAGES) + 2048;
        const int limit = want < optin ? want : optin;
        e = cudaFuncSetAttribute(kernel_of<T, CW>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 limit);
        if (e != cudaSuccess) return e;
        info.prepared[prec_of<T>()][vi] = true;
    }
    return cudaSuccess;
}

template <typename T, int CW>
cudaError_t plan_for(int stages, int ctas_per_sm, int hint, StagedPlan *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (stages < 2 || stages > MAX_STAGES) return cudaErrorInvalidValue;
    if ((e = prepare<T, CW>(dev)) != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of<T, CW>(),
                                                      (CW + 1) * 32, smem_bytes<T, CW>(stages));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    out->stages = stages;
    out->ctas_per_sm = per_sm;
    out->grid = g_info[dev].sms * per_sm;
    out->consumer_warps = CW;
    out->hint = hint ? 1 : 0;
    return cudaSuccess;
}

template <typename T, int CW>
cudaError_t launch_cw(const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                      const Coef<typename Store<T>::C> &k, int *status, const StagedPlan &plan,
                      int *blocks_out, cudaStream_t stream) {
    const long long plane = (long long)nx * ny;
    const long long n_tiles = (long long)(nx / tile_width<T, CW>()) * ny;
    const int grid = (int)(n_tiles < plan.grid ? n_tiles : plan.grid);
    const size_t smem = smem_bytes<T, CW>(plan.stages);
    if (blocks_out) *blocks_out = grid;
    step_staged<T, CW><<<grid, (CW + 1) * 32, smem, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                             bc_y, plan.stages, plan.hint, k,
                                                             status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plan_t(int stages, int ctas_per_sm, int cw, int hint, StagedPlan *out) {
    return cw == 4 ? plan_for<T, 4>(stages, ctas_per_sm, hint, out)
                   : plan_for<T, 8>(stages, ctas_per_sm, hint, out);
}

}  // namespace

int staged_tile_width(int precision, int consumer_warps) {
    const int v = precision == PREC_FP32 ? 4 : precision == PREC_FP64 ? 2 : 8;
    return consumer_warps * 32 * v;
}

bool staged_supported(int precision, int nx, int ny, int consumer_warps) {
    if (consumer_warps != 4 && consumer_warps != 8) return false;
    // 16-bit storage is kept relative to tile references (refs16.cuh), which
    // the vector kernels handle; this kernel keeps FP32 and FP64 storage
    if (precision != PREC_FP32 && precision != PREC_FP64) return false;
    const int w = staged_tile_width(precision, consumer_warps);
    return ny >= 1 && nx >= w && nx % w == 0;
}

cudaError_t staged_plan(int precision, int stages, int ctas_per_sm, int consumer_warps,
                        int l2_hint, StagedPlan *out) {
    if (stages <= 0) stages = 2;
    if (consumer_warps <= 0) consumer_warps = 8;
    if (consumer_warps != 4 && consumer_warps != 8) return cudaErrorInvalidValue;
    switch (precision) {
        case PREC_FP32: return plan_t<float>(stages, ctas_per_sm, consumer_warps, l2_hint, out);
        case PREC_FP64: return plan_t<double>(stages, ctas_per_sm, consumer_warps, l2_hint, out);
        default: return cudaErrorNotSupported;     // 16-bit storage: the vector kernels
    }
}

template <typename T>
cudaError_t launch_step_staged(const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                               const Coef<typename Store<T>::C> &k, int *status,
                               const StagedPlan &plan, int *blocks_out, cudaStream_t stream) {
    if (plan.consumer_warps == 4)
        return launch_cw<T, 4>(src, dst, nx, ny, bc_x, bc_y, k, status, plan, blocks_out, stream);
    return launch_cw<T, 8>(src, dst, nx, ny, bc_x, bc_y, k, status, plan, blocks_out, stream);
}

// One thread waits, with the kernel's bounded wait, on a fresh mbarrier
// that no thread ever arrives at: the wait gives up after its clock limit
// (about 2 s) and sets *status, exactly as a stalled pipeline stage would.
__global__ void wait_probe(int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) stage_wait(&bar, 0u, status);
}

cudaError_t launch_wait_probe(int *status, cudaStream_t stream) {
    wait_probe<<<1, 32, 0, stream>>>(status);
    return cudaGetLastError();
}

#define PLBM_STAGED(T)                                                                       \
    template cudaError_t launch_step_staged<T>(const T *, T *, int, int, int, int,           \
                                               const Coef<Store<T>::C> &, int *,             \
                                               const StagedPlan &, int *, cudaStream_t);
PLBM_STAGED(float)
PLBM_STAGED(double)

}  // namespace plbm
