// Plain time steps for 16-bit storage, pipelined: a persistent grid whose
// threads each walk a sequence of 16-byte vectors (8 nodes of one row, one
// tile of the tile references of refs16.cuh) and, while one is being
// collided, already have the next one's data on its way into shared memory
// (cp.async: no registers hold data in flight).
//
// The step is the one of the node-pair kernels (pairs16.cuh): pull with the
// x shift on packed words and the neighbour word from the adjacent lane
// (Eq. 13, left-hand side; seam jump of Eqs. 59-60 at the row ends), the
// walls of Eq. 58, the collision of Eqs. 15, 16, 53-54 on node pairs, and
// the storage relative to the tile references, with the same operations in
// the same order: the same bits as every other kernel.
//
// Why: with the tile references the node-pair collision needs about 116
// registers per thread.  One thread per vector then fits 16 warps per SM
// without spilling, too few for its loads alone to keep HBM busy; squeezed
// to 24 warps it spills ~150 bytes per thread.  Here each thread's next
// vector (its 8 plane vectors, the two edge words and its tile's
// references: 192 bytes) is in flight in shared memory while it computes.
//
// Per thread and iteration: wait for its copies, read them into registers,
// shift (shuffles), issue the copies of the vector STAGES iterations ahead
// into the same shared slots, then collide and store.  Every thread reads and writes only
// its own slots, so no block barrier is needed; the slots of a stage are
// refilled only after the values read from them have been consumed.
#include <type_traits>

#include "lbm_kernels.h"
#include "pairs16.cuh"
#include "vector_pull.cuh"

namespace plbm {
namespace {

// shared-memory slots (16 bytes each) per thread: 8 plane vectors, 2 edge
// words per plane (planes 0-3, 4-7), the tile's own reference record, the
// stored-against references of the tiles above and below, and for lanes at a
// warp edge or a row end those of the neighbouring tiles (left | right in
// rows y, y - 1, y + 1)
#ifndef PLBM_P16_THREADS
#define PLBM_P16_THREADS 256
#endif
#ifndef PLBM_P16_STAGES
#define PLBM_P16_STAGES 1
#endif
constexpr int SLOTS = 15;
constexpr int STAGES = PLBM_P16_STAGES;     // vectors in flight per thread
constexpr int THREADS = PLBM_P16_THREADS;

__device__ __forceinline__ uint32_t s_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s_addr(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s_addr(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s_addr(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}
// waits until at most N of this thread's newest copy groups are pending
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Where vector t of the lattice is and which neighbours its lane loads.
struct VPos {
    int y, xv, x0;
    bool active, bottom, top, need_left, need_right;
};
__device__ __forceinline__ VPos vpos(long long t, long long total, int tpr, int ny, bool walls,
                                     int lane) {
    VPos p;
    p.active = t < total;
    p.y = p.active ? int(t / tpr) : 0;
    p.xv = p.active ? int(t - (long long)p.y * tpr) : 0;
    p.x0 = p.xv * 8;
    p.bottom = walls && p.y == 0;
    p.top = walls && p.y == ny - 1;
    p.need_left = (lane == 0 || p.xv == 0) && p.active;
    p.need_right = (lane == 31 || p.xv + 1 == tpr) && p.active;
    return p;
}

#ifndef PLBM_P16_BLOCKS
#define PLBM_P16_BLOCKS 2
#endif

template <typename T, bool SR>
__global__ void __launch_bounds__(THREADS, PLBM_P16_BLOCKS)
step_pipe16(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny, long long plane,
            int bc_x, int bc_y, Coef<float> k) {
    extern __shared__ uint4 slots[];        // [STAGES][SLOTS][THREADS]
    const int tid = threadIdx.x, lane = tid & 31;
    const int tpr = nx / 8;
    const long long total = (long long)tpr * ny;
    const long long chunks = (total + THREADS - 1) / THREADS;
    const bool walls = bc_y == BC_WALLS, grad = bc_x == BC_GRADIENT;

    // copies of vector p into stage st (all of them land in this thread's slots)
    auto issue = [&](const VPos &p, int st) {
        if (!p.active) return;
        uint4 *my = slots + (size_t)st * SLOTS * THREADS + tid;
        const int sx_left = p.x0 == 0 ? nx - 1 : p.x0 - 1;
        const int sx_right = p.x0 + 8 >= nx ? p.x0 + 8 - nx : p.x0 + 8;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int cx = cx_of(i), cy = cy_of(i);
            int sy = p.y - cy;
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            const bool unknown = (cy > 0 && p.bottom) || (cy < 0 && p.top);
            if (unknown) continue;
            const T *row = src + (long long)i * plane + (long long)sy * nx;
            cp_async16(my + i * THREADS, row + p.x0);
            // the neighbour value travels in the aligned 4-byte word that
            // holds it: (sx - 1, sx) on the left (sx odd), (sx, sx + 1) on
            // the right (sx even); word i & 3 of slot 8 + i / 4
            unsigned *edge = reinterpret_cast<unsigned *>(my + (8 + (i >> 2)) * THREADS) + (i & 3);
            if (cx > 0 && p.need_left) cp_async4(edge, row + sx_left - 1);
            if (cx < 0 && p.need_right) cp_async4(edge, row + sx_right);
        }
        const long long ym = p.y == 0 ? ny - 1 : p.y - 1, yp = p.y + 1 == ny ? 0 : p.y + 1,
                        y0 = p.y;
        cp_async16(my + 10 * THREADS, src + ref_at(k, y0 * tpr + p.xv));
        cp_async8(my + 11 * THREADS, src + ref_at(k, ym * tpr + p.xv));
        cp_async8(reinterpret_cast<char *>(my + 11 * THREADS) + 8,
                  src + ref_at(k, yp * tpr + p.xv));
        if (p.need_left) {
            const int xl = p.xv == 0 ? tpr - 1 : p.xv - 1;
            cp_async8(my + 12 * THREADS, src + ref_at(k, y0 * tpr + xl));
            cp_async8(my + 13 * THREADS, src + ref_at(k, ym * tpr + xl));
            cp_async8(my + 14 * THREADS, src + ref_at(k, yp * tpr + xl));
        }
        if (p.need_right) {
            const int xr = p.xv + 1 == tpr ? 0 : p.xv + 1;
            cp_async8(reinterpret_cast<char *>(my + 12 * THREADS) + 8,
                      src + ref_at(k, y0 * tpr + xr));
            cp_async8(reinterpret_cast<char *>(my + 13 * THREADS) + 8,
                      src + ref_at(k, ym * tpr + xr));
            cp_async8(reinterpret_cast<char *>(my + 14 * THREADS) + 8,
                      src + ref_at(k, yp * tpr + xr));
        }
    };

    long long c = blockIdx.x;
    if (c >= chunks) return;
    const long long stride = gridDim.x;
    // prologue: the first STAGES vectors in flight, one copy group each
    VPos cur = vpos(c * THREADS + tid, total, tpr, ny, walls, lane);
    issue(cur, 0);
    cp_async_commit();
#pragma unroll
    for (int s = 1; s < STAGES; ++s) {
        const long long cs = c + s * stride;
        if (cs < chunks) issue(vpos(cs * THREADS + tid, total, tpr, ny, walls, lane), s);
        cp_async_commit();
    }
    int st = 0;
    for (; c < chunks; c += stride) {
        const long long t = c * THREADS + tid;
        uint4 *my = slots + (size_t)st * SLOTS * THREADS + tid;
        cp_async_wait<STAGES - 1>();     // this vector's group has landed
        // this vector's data, from the slots
        uint4 w[8];
        unsigned edge[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int cy = cy_of(i);
            const bool unknown = (cy > 0 && cur.bottom) || (cy < 0 && cur.top);
            w[i] = (cur.active && !unknown) ? my[i * THREADS] : make_uint4(0u, 0u, 0u, 0u);
        }
        {
            const uint4 e0 = my[8 * THREADS], e1 = my[9 * THREADS];
            edge[0] = e0.x; edge[1] = e0.y; edge[2] = e0.z; edge[3] = e0.w;
            edge[4] = e1.x; edge[5] = e1.y; edge[6] = e1.z; edge[7] = e1.w;
        }
        VecRefWords rw;
        rw.own = my[10 * THREADS];
        {
            const uint4 ud = my[11 * THREADS];
            rw.up = make_uint2(ud.x, ud.y);
            rw.dn = make_uint2(ud.z, ud.w);
        }
        // the neighbouring tiles' references (only lanes at a warp edge or a
        // row end copied them; the others' are not used)
        {
            const uint4 a = my[12 * THREADS], b = my[13 * THREADS], c3 = my[14 * THREADS];
            rw.l0 = make_uint2(a.x, a.y);
            rw.r0 = make_uint2(a.z, a.w);
            rw.lu = make_uint2(b.x, b.y);
            rw.ru = make_uint2(b.z, b.w);
            rw.ld = make_uint2(c3.x, c3.y);
            rw.rd = make_uint2(c3.z, c3.w);
        }
        // x shift on the packed words (Eq. 13, left-hand side)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int cx = cx_of(i);
            if (cx > 0) {
                unsigned nb = __shfl_up_sync(0xffffffffu, w[i].w, 1);
                if (cur.need_left) nb = edge[i];            // its high half is the value
                w[i] = shift_from_left(w[i], nb);
            } else if (cx < 0) {
                unsigned nb = __shfl_down_sync(0xffffffffu, w[i].x, 1);
                if (cur.need_right) nb = edge[i];           // its low half is the value
                w[i] = shift_from_right(w[i], nb);
            }
        }
        float Rd[8], Rx[8];
        uint2 enc;
        vector_ref_pops<T>(rw, k, cur.need_left, cur.need_right, Rd, Rx, enc);
        // every value read from the slots is consumed: refill them with the
        // data of the vector STAGES iterations ahead
        const long long cn = c + STAGES * stride;
        if (cn < chunks) issue(vpos(cn * THREADS + tid, total, tpr, ny, walls, lane), st);
        cp_async_commit();
        pull_edge_refs(Rd, Rx, cur.need_left, cur.need_right);
        if (cur.active) {
            const SeamAdd seam{cur.need_left, cur.x0 == 0 && grad, cur.need_right,
                               cur.x0 + 8 == nx && grad};
            float sums[3];
            float Re[8];
            ref_pops(ref_of<T>(enc), k, Re);
            const long long out = (long long)cur.y * nx + cur.x0;
            collide_words16<T, SR>(w, k, seam, cur.bottom, cur.top, Rd, Rx, Re, sums,
                                   (unsigned)(out >> 1));
#pragma unroll
            for (int i = 0; i < 8; ++i) st_stream(dst + (long long)i * plane + out, w[i]);
            st_ref(dst, k, t, enc, next_ref<T>(sums[0], sums[1], sums[2], k, k.ref_gamma));
        }
        cur = vpos((c + stride) * THREADS + tid, total, tpr, ny, walls, lane);
        st = st + 1 == STAGES ? 0 : st + 1;
    }
    cp_async_wait_all();
}

constexpr size_t SMEM = (size_t)STAGES * SLOTS * THREADS * sizeof(uint4);

struct Prep {
    bool ready = false;
    int grid = 0;
};
Prep g_prep[64][2][2];      // device, storage kind, rounding

template <typename T> constexpr int kind_of() { return std::is_same<T, __half>::value ? 0 : 1; }

template <typename T, bool SR>
cudaError_t prepare_t(int dev) {
    Prep &p = g_prep[dev][kind_of<T>()][SR ? 1 : 0];
    if (p.ready) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(step_pipe16<T, SR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_pipe16<T, SR>, THREADS,
                                                      SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.grid = sms * per_sm;
    p.ready = true;
    return cudaSuccess;
}

}  // namespace

cudaError_t prepare_pipe16(int precision) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (precision == PREC_FP16) {
        if ((e = prepare_t<__half, false>(dev)) != cudaSuccess) return e;
        return prepare_t<__half, true>(dev);
    }
    if (precision == PREC_BF16) {
        if ((e = prepare_t<__nv_bfloat16, false>(dev)) != cudaSuccess) return e;
        return prepare_t<__nv_bfloat16, true>(dev);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_step_pipe16(const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                               const Coef<float> &k, cudaStream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const bool sr = k.stochastic != 0;
    const Prep &p = g_prep[dev][kind_of<T>()][sr ? 1 : 0];
    if (!p.ready) return cudaErrorNotReady;      // prepare_pipe16 was not called on this device
    const long long chunks = ((long long)(nx / 8) * ny + THREADS - 1) / THREADS;
    const int grid = (int)(chunks < p.grid ? chunks : p.grid);
    if (sr)
        step_pipe16<T, true><<<grid, THREADS, SMEM, stream>>>(src, dst, nx, ny,
                                                              (long long)nx * ny, bc_x, bc_y, k);
    else
        step_pipe16<T, false><<<grid, THREADS, SMEM, stream>>>(src, dst, nx, ny,
                                                               (long long)nx * ny, bc_x, bc_y, k);
    return cudaGetLastError();
}

template cudaError_t launch_step_pipe16<__half>(const __half *, __half *, int, int, int, int,
                                                const Coef<float> &, cudaStream_t);
template cudaError_t launch_step_pipe16<__nv_bfloat16>(const __nv_bfloat16 *, __nv_bfloat16 *,
                                                       int, int, int, int, const Coef<float> &,
                                                       cudaStream_t);

}  // namespace plbm
