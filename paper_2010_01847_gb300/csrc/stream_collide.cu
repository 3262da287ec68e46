// Fused pull-stream + boundary + collision kernels: one launch is one time
// step of Eq. 13 over the whole lattice.
//
// The kernels read the post-collision planes of step n-1 (`src`), pull the
// populations arriving at each node (left-hand side of Eq. 13, seam jump of
// Eqs. 59-60, diffuse walls of Eq. 58), collide them in registers
// (Eqs. 15, 16, 53, 54) and write the post-collision planes of step n
// (`dst`).  Layout: structure of arrays, 8 planes of ny*nx, x fastest.
// With RES the kernel also accumulates the residual sums of the pulled state
// (the state at step n) and writes one set of 5 partial sums per block.
#include <type_traits>

#include "lbm_kernels.h"
#include "pairs16.cuh"
#include "vector_pull.cuh"

namespace plbm {

// ---------------------------------------------------------------------------
// Scalar kernel: one thread per node, any nx.  Serves ragged lattices (nx not
// a multiple of the vector width) and is the simplest statement of the step.
template <typename T, bool RES>
__global__ void __launch_bounds__(256)
step_scalar(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny,
            long long plane, int bc_x, int bc_y, Coef<typename Store<T>::C> k,
            ResidualReq<typename Store<T>::C> rq) {
    using C = typename Store<T>::C;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    C loc[5] = {C(0), C(0), C(0), C(0), C(0)};
    if (node < plane) {
        const int y = int(node / nx);
        const int x = int(node - (long long)y * nx);
        C d[8];
        pull_node<T>(src, plane, nx, ny, x, y, bc_x, bc_y, k, d);
        if (RES) residual_node(d, k, rq.inv_scale, rq.prev, plane, node, rq.have_prev != 0, loc);
        collide(d, k);
#pragma unroll
        for (int i = 0; i < 8; ++i) dst[(long long)i * plane + node] = Store<T>::put(d[i]);
    }
    if (RES) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        warp_flush_residual(loc, acc);
        block_sum5_lane0(acc, rq.partials + (size_t)blockIdx.x * 5);
    }
}

// The scalar kernel for 16-bit storage (populations stored relative to tile
// references, refs16.cuh).  Tiles of 8 nodes are 8 aligned lanes, whose sums
// go through shuffles, so every lane of the warp runs the step: lanes past
// the lattice's end (whole tiles, as nx is a multiple of 8 then) work on the
// last node and store nothing.
template <typename T, bool RES, bool SR>
__global__ void __launch_bounds__(256)
step_scalar16(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny, long long plane,
              int bc_x, int bc_y, Coef<float> k, ResidualReq<float> rq) {
    static_assert(sizeof(T) == 2, "16-bit storage");
    const long long at = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = at < plane;
    const long long node = valid ? at : plane - 1;
    const int y = int(node / nx);
    const int x = int(node - (long long)y * nx);
    float loc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float d[8];
    pull_node<T>(src, plane, nx, ny, x, y, bc_x, bc_y, k, d);
    if (RES && valid) residual_node(d, k, rq.inv_scale, rq.prev, plane, node, rq.have_prev != 0, loc);
    float rho, mx, my;
    moments_f32(d, rho, mx, my);
    relax_f32(d, rho, mx, my, k);
    const long long tile = tile_of(k, x, y);
    const uint4 both = ld_ref_both(src, k, tile);
    const uint2 enc = make_uint2(both.z, both.w);
    float Re[8];
    ref_pops(ref_of<T>(enc), k, Re);
    // stored as node pairs (2p, 2p + 1) like the vector kernels: with
    // stochastic rounding both lanes of a pair form the pair's random bits
    // (lane parity = node parity: blocks hold whole warps)
    const bool odd = node & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float v = f_sub(d[i], Re[i]);
        const float o = SR ? __shfl_xor_sync(0xffffffffu, v, 1) : 0.f;
        const unsigned wd = store_word<T, SR>(odd ? make_float2(o, v) : make_float2(v, o),
                                              (unsigned)(node >> 1), i);
        if (valid)
            reinterpret_cast<unsigned short *>(dst)[(long long)i * plane + node] =
                (unsigned short)(odd ? wd >> 16 : wd & 0xffffu);
    }
    if (k.tile_shift == 3) {
        rho = tile_tree_lanes(rho);
        mx = tile_tree_lanes(mx);
        my = tile_tree_lanes(my);
    }
    if (valid && (x & ((1 << k.tile_shift) - 1)) == 0)
        st_ref(dst, k, tile, enc, next_ref<T>(rho, mx, my, k, k.ref_gamma));
    if (RES) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        warp_flush_residual(loc, acc);
        block_sum5_lane0(acc, rq.partials + (size_t)blockIdx.x * 5);
    }
}

// ---------------------------------------------------------------------------
// Vector kernel: each thread owns V consecutive nodes of one row and moves
// every plane with one aligned 16-byte load and one 16-byte store.  The
// x-shifted populations (c_x = +-1) take their out-of-vector neighbour from
// the adjacent lane by a warp shuffle; the first/last lane of a warp, and
// rows' ends, load that one element directly (wrapping at the seam).
// Requires nx % V == 0.  Threads are laid out row-major over the lattice,
// so a warp may straddle two rows; the row test handles that.
//
// Occupancy: the kernel is latency-bound on its loads, so it is compiled for
// as many resident 256-thread blocks per SM as the register file allows
// without heavy spilling (FP32: 5 blocks = 48 registers, 16 bytes spilled;
// measured 6.73 TB/s at 8192^2 against 6.29 TB/s at 4 blocks / 54 registers;
// the residual step at 4 blocks = 64 registers costs 560 us over a plain step
// against 680 us at 3 blocks, despite spilling 68 bytes).
template <typename T> struct VecMinBlocks { static constexpr int plain = 3, res = 2; };
template <> struct VecMinBlocks<float> { static constexpr int plain = 5, res = 4; };
template <> struct VecMinBlocks<double> { static constexpr int plain = 4, res = 3; };

// SIDES: the instantiation for lattices with a BC_SIDES direction (the
// per-side treatments of Section 2.5 after the pull, as in pull_node); the
// others never see the side logic.
template <typename T, bool RES, bool SIDES = false, bool SR = false>
__global__ void __launch_bounds__(256, RES ? VecMinBlocks<T>::res : VecMinBlocks<T>::plain)
step_vector(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny,
            long long plane, int bc_x, int bc_y, Coef<typename Store<T>::C> k,
            ResidualReq<typename Store<T>::C> rq) {
    using C = typename Store<T>::C;
    constexpr int V = Pack<T>::V;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    C d[8][V];
    uint2 enc = make_uint2(0u, 0u);       // 16-bit storage: the tile's next reference
    const VecPos p = vector_pull<T, SIDES>(src, nx, ny, plane, bc_x, bc_y, k, t, d, &enc);
    const int y = p.y, x0 = p.x0;
    // the wall rows of Eq. 58 (with SIDES, p.bottom/p.top also flag y sides)
    const bool walls = !SIDES || bc_y == BC_WALLS;
    const bool active = p.active, bottom = p.bottom && walls, top = p.top && walls;
    const bool open_x = SIDES && bc_x == BC_SIDES, open_y = SIDES && bc_y == BC_SIDES;

    C loc[5] = {C(0), C(0), C(0), C(0), C(0)};
    if (active) {
        const long long out = (long long)y * nx + x0;
        C n[V][8];
#pragma unroll
        for (int j = 0; j < V; ++j) {
#pragma unroll
            for (int i = 0; i < 8; ++i) n[j][i] = d[i][j];
            if (bottom) wall_bottom(n[j], k);
            if (top) wall_top(n[j], k);
            if (SIDES && (open_x || open_y))
                apply_sides(n[j], k, open_x && x0 + j == 0, open_x && x0 + j == nx - 1,
                            open_y && y == 0, open_y && y == ny - 1);
        }
        if (RES) residual_vec<C, V>(n, k, rq.inv_scale, rq.prev, plane, out, rq.have_prev != 0,
                                    loc);
        if constexpr (sizeof(T) == 2) {
            collide_store16<T, SR>(n, k, dst, plane, out, t, enc);     // tile t = vector t
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                collide(n[j], k);
#pragma unroll
                for (int i = 0; i < 8; ++i) d[i][j] = n[j][i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                st_stream(dst + (long long)i * plane + out, Pack<T>::pack(d[i]));
        }
    }
    if (RES) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        warp_flush_residual(loc, acc);
        block_sum5_lane0(acc, rq.partials + (size_t)blockIdx.x * 5);
    }
}

// ---------------------------------------------------------------------------
// Vector kernel for 16-bit storage, plain steps on periodic / gradient /
// wall lattices: the step of step_vector with the node pairs of
// pairs16.cuh.  The x shift runs on the packed words (the neighbour's word
// from the adjacent lane, or at a warp edge or a row end the one element
// loaded directly); the collision runs two nodes per packed FP32 pair
// instruction, half the instructions of the node-by-node form, with the
// same bits.  Inputs stay packed until their pair is needed, so the kernel
// fits 4 blocks of 256 threads per SM (the node-by-node form: 3).
namespace {

__device__ __forceinline__ unsigned ld_u16(const void *p) {
    unsigned short r;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return r;
}

}  // namespace

// Resident 256-thread blocks per SM the node-pair residual step is compiled
// for (registers per thread = 65536 / (256 x blocks)); the plain 16-bit
// steps run the pipelined kernel of pipe16.cu.
#ifndef PLBM_V16_RES_BLOCKS
#define PLBM_V16_RES_BLOCKS 2
#endif

// The 16-bit step that also reduces the residual of the pulled state (one
// step in many): one thread per 16-byte vector, the node pairs of
// pairs16.cuh with the tile references, residual_terms on each node in node
// order (the history planes read and written as node pairs): the sums the
// node-by-node kernel forms.
template <typename T, bool SR>
__global__ void __launch_bounds__(256, PLBM_V16_RES_BLOCKS)
step_vector16_res(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny,
                  long long plane, int bc_x, int bc_y, Coef<float> k, ResidualReq<float> rq) {
    static_assert(sizeof(T) == 2 && Pack<T>::V == 8, "16-bit storage");
    constexpr int V = 8;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int tpr = nx / V;
    const long long total = (long long)tpr * ny;
    const bool active = t < total;
    const int y = active ? int(t / tpr) : 0;
    const int xv = active ? int(t - (long long)y * tpr) : 0;
    const int x0 = xv * V;
    const int lane = threadIdx.x & 31;
    const bool walls = bc_y == BC_WALLS;
    const bool bottom = walls && y == 0;
    const bool top = walls && y == ny - 1;
    const bool need_left = (lane == 0 || xv == 0) && active;
    const bool need_right = (lane == 31 || xv + 1 == tpr) && active;
    const int sx_left = x0 == 0 ? nx - 1 : x0 - 1;
    const int sx_right = x0 + V >= nx ? x0 + V - nx : x0 + V;

    const VecRefWords rw = vector_ref_loads<T>(src, k, ny, y, xv, need_left, need_right);
    uint4 w[8];
    unsigned edge[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        int sy = y - cy;
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        const long long row = (long long)i * plane + (long long)sy * nx;
        const bool unknown = (cy > 0 && bottom) || (cy < 0 && top);
        w[i] = (active && !unknown) ? ld_stream(src + row + x0) : make_uint4(0u, 0u, 0u, 0u);
        edge[i] = 0u;
        if (cx > 0 && need_left && !unknown) edge[i] = ld_u16(src + row + sx_left);
        if (cx < 0 && need_right && !unknown) edge[i] = ld_u16(src + row + sx_right);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i);
        if (cx > 0) {
            unsigned nb = __shfl_up_sync(0xffffffffu, w[i].w, 1);
            if (need_left) nb = edge[i] << 16;
            w[i] = shift_from_left(w[i], nb);
        } else if (cx < 0) {
            unsigned nb = __shfl_down_sync(0xffffffffu, w[i].x, 1);
            if (need_right) nb = edge[i];
            w[i] = shift_from_right(w[i], nb);
        }
    }
    float Rd[8], Rx[8];
    uint2 enc;
    vector_ref_pops<T>(rw, k, need_left, need_right, Rd, Rx, enc);
    pull_edge_refs(Rd, Rx, need_left, need_right);
    float loc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (active) {
        const bool grad = bc_x == BC_GRADIENT;
        const SeamAdd seam{need_left, x0 == 0 && grad, need_right, x0 + V == nx && grad};
        const long long out = (long long)y * nx + x0;
        const bool have_prev = rq.have_prev != 0;
        // the thread's 8 nodes of each history plane, read and written as
        // 16-byte vectors around the collision (reading and writing them a
        // pair at a time in between, each store invalidated the L1 line the
        // next pair's load needed: 3x the step's time)
        float h[3][8];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (have_prev) {
                load_cvec<float, 8>(rq.prev + q * plane + out, h[q]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) h[q][j] = 0.f;
            }
        }
        auto residual = [&](int m, const float2 (&f)[8]) {
            float n0[8], n1[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                n0[i] = f[i].x;
                n1[i] = f[i].y;
            }
            residual_terms(n0, k, rq.inv_scale, h[0][2 * m], h[1][2 * m], h[2][2 * m], have_prev,
                           loc);
            residual_terms(n1, k, rq.inv_scale, h[0][2 * m + 1], h[1][2 * m + 1],
                           h[2][2 * m + 1], have_prev, loc);
        };
        float sums[3];
        float Re[8];
        ref_pops(ref_of<T>(enc), k, Re);
        collide_words16<T, SR>(w, k, seam, bottom, top, Rd, Rx, Re, sums, (unsigned)(out >> 1),
                               residual);
#pragma unroll
        for (int q = 0; q < 3; ++q) store_cvec<float, 8>(rq.prev + q * plane + out, h[q]);
#pragma unroll
        for (int i = 0; i < 8; ++i) st_stream(dst + (long long)i * plane + out, w[i]);
        st_ref(dst, k, t, enc, next_ref<T>(sums[0], sums[1], sums[2], k, k.ref_gamma));
    }
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    warp_flush_residual(loc, acc);
    block_sum5_lane0(acc, rq.partials + (size_t)blockIdx.x * 5);
}

// ---------------------------------------------------------------------------
// Threads per block of a step launch: 256, or fewer (a multiple of 32) when
// the lattice is small, so that the launch still spreads over every SM: a
// small lattice is latency-bound, and FP64 arithmetic runs at about one
// operation per clock per SM on this GPU (the 128 x 32 FP64 channel would
// otherwise run on 8 of the 152 SMs).
int step_block_size(long long threads) {
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        dev = 0;
    }
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            v <= 0) {
            (void)cudaGetLastError();
            v = 152;
        }
        sms[dev] = v;
    }
    const long long per_sm = (threads + sms[dev] - 1) / sms[dev];
    if (per_sm >= 256) return 256;
    return (int)(per_sm <= 32 ? 32 : (per_sm + 31) / 32 * 32);
}

template <typename T>
cudaError_t launch_step(int kernel, const T *src, T *dst, int nx, int ny, int bc_x, int bc_y,
                        const Coef<typename Store<T>::C> &k, int *status,
                        const ResidualReq<typename Store<T>::C> *rq, const StagedPlan &plan,
                        int *blocks_out, cudaStream_t stream) {
    const long long plane = (long long)nx * ny;
    // a step that also reduces the residual (one step in many) runs on the
    // vector kernel, whose warps read the history planes with 16-byte vectors
    if (kernel == KERNEL_STAGED && rq) kernel = KERNEL_VECTOR;
    // single steps of a cluster-resident lattice (the residual step) run on
    // the vector kernel when nx allows, else the scalar one
    // and so do the single steps of a multi-step (wave) lattice
    if (kernel == KERNEL_RESIDENT || kernel == KERNEL_WAVE)
        kernel = nx % Pack<T>::V == 0 ? KERNEL_VECTOR : KERNEL_SCALAR;
    if constexpr (sizeof(T) == 2) {
        // the staged kernel keeps FP32 / FP64 storage only (16-bit storage
        // with tile references runs on the vector kernels)
        if (kernel == KERNEL_STAGED) return cudaErrorNotSupported;
    } else {
        if (kernel == KERNEL_STAGED)
            return launch_step_staged<T>(src, dst, nx, ny, bc_x, bc_y, k, status, plan,
                                         blocks_out, stream);
    }
    const ResidualReq<typename Store<T>::C> none{};
    const long long threads = kernel == KERNEL_VECTOR ? plane / Pack<T>::V : plane;
    const int bs = step_block_size(threads);
    const unsigned blocks = (unsigned)((threads + bs - 1) / bs);
    if (blocks_out) *blocks_out = (int)blocks;
    const bool sides = bc_x == BC_SIDES || bc_y == BC_SIDES;
    if constexpr (sizeof(T) == 2) {
        // 16-bit storage: the kernels of the chosen rounding (refs16.cuh)
        auto run16 = [&](auto sr_tag) {
            constexpr bool SR = decltype(sr_tag)::value;
            if (kernel == KERNEL_VECTOR && sides) {
                if (rq)
                    step_vector<T, true, true, SR><<<blocks, bs, 0, stream>>>(
                        src, dst, nx, ny, plane, bc_x, bc_y, k, *rq);
                else
                    step_vector<T, false, true, SR><<<blocks, bs, 0, stream>>>(
                        src, dst, nx, ny, plane, bc_x, bc_y, k, none);
            } else if (kernel == KERNEL_VECTOR) {
                if (!rq) return launch_step_pipe16<T>(src, dst, nx, ny, bc_x, bc_y, k, stream);
                step_vector16_res<T, SR><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane,
                                                                    bc_x, bc_y, k, *rq);
            } else if (rq) {
                step_scalar16<T, true, SR><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane,
                                                                      bc_x, bc_y, k, *rq);
            } else {
                step_scalar16<T, false, SR><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane,
                                                                       bc_x, bc_y, k, none);
            }
            return cudaGetLastError();
        };
        return k.stochastic ? run16(std::true_type{}) : run16(std::false_type{});
    } else {
        if (kernel == KERNEL_VECTOR && sides) {
            if (rq)
                step_vector<T, true, true><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane,
                                                                      bc_x, bc_y, k, *rq);
            else
                step_vector<T, false, true><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane,
                                                                       bc_x, bc_y, k, none);
        } else if (kernel == KERNEL_VECTOR) {
            if (rq)
                step_vector<T, true><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                                bc_y, k, *rq);
            else
                step_vector<T, false><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                                 bc_y, k, none);
        } else {
            if (rq)
                step_scalar<T, true><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                                bc_y, k, *rq);
            else
                step_scalar<T, false><<<blocks, bs, 0, stream>>>(src, dst, nx, ny, plane, bc_x,
                                                                 bc_y, k, none);
        }
    }
    return cudaGetLastError();
}

long long step_blocks(int kernel, int precision, int nx, int ny, const StagedPlan &plan) {
    const long long plane = (long long)nx * ny;
    (void)plan;
    if (kernel == KERNEL_STAGED) kernel = KERNEL_VECTOR;    // residual steps run there
    if (kernel == KERNEL_RESIDENT || kernel == KERNEL_WAVE)
        kernel = nx % vector_width(precision) == 0 ? KERNEL_VECTOR : KERNEL_SCALAR;
    const long long threads = kernel == KERNEL_VECTOR ? plane / vector_width(precision) : plane;
    const int bs = step_block_size(threads);
    return (threads + bs - 1) / bs;
}

int vector_width(int precision) {
    switch (precision) {
        case PREC_FP32: return Pack<float>::V;
        case PREC_FP64: return Pack<double>::V;
        default: return Pack<__half>::V;
    }
}

#define PLBM_STEP(T)                                                                         \
    template cudaError_t launch_step<T>(int, const T *, T *, int, int, int, int,             \
                                        const Coef<Store<T>::C> &, int *,                    \
                                        const ResidualReq<Store<T>::C> *, const StagedPlan &, \
                                        int *, cudaStream_t);
PLBM_STEP(float)
PLBM_STEP(double)
PLBM_STEP(__half)
PLBM_STEP(__nv_bfloat16)

}  // namespace plbm
