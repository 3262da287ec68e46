// The multi-step stream-collide kernel for 16-bit storage (FP16 / BF16
// deviations relative to tile reference equilibria, refs16.cuh): K time
// steps per launch with the strip march of wave.cuh.
//
// Level 0 decodes the source rows as every 16-bit kernel does: the stored
// value plus the reference population R_i of its tile's stored-against
// reference.  Levels 1..K-1 stay in FP32 registers.  Level K is stored
// against the reference of its tile worked out one step before (level
// K - 1: {rho, gamma m} / 32 from the tile sums of the pulled moments, the
// one-step lag of the single-step kernels) and writes the tile's record
// {that reference, the next one from level K's sums}.  So a launch rounds to
// 16 bits once per K steps instead of once per step: its result is not the
// bits of K single 16-bit steps (it is closer to the exact one), and the
// storage format between launches is the same, so every other kernel and
// read-out continues from it.
//
// Tiles are the 8 nodes of a row from x = 8t; a lane's node pair (xa, xa + 1)
// lies in one tile and 4 consecutive lanes hold a tile, the lane o
// positions into it; strips have a halo of 4 columns whatever K (<= 4), so
// that the 56 columns a strip writes are 7 whole tiles.  Tile sums use the
// tree ((0 + 2) + (4 + 6)) + ((1 + 3) + (5 + 7)) of the single-step
// kernels.  Requires nx % 8 == 0.
#include "lbm_kernels.h"
#include "refs16.cuh"
#include "wave.cuh"

namespace plbm {
namespace {

using wave::mod3;

constexpr int W16_WARPS = 1;          // one strip per block, as the FP32 kernel
constexpr int W16_RING = 4;
// one ring slot: 8 planes x 32 lanes of one 32-bit word (the lane's node
// pair), then 32 lanes x 8 bytes of stored-against reference
constexpr int W16_SLOT_WORDS = 8 * 32 + 32 * 2;
constexpr int W16_SMEM = W16_WARPS * W16_RING * W16_SLOT_WORDS * 4;

struct Strip16 {
    const void *src;
    void *dst;
    long long plane;
    int nx, ny, bc_x, bc_y, seg_rows;
};

__device__ __forceinline__ void cp_async4(unsigned *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8w(unsigned *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void st_word(void *p, unsigned v) {
    asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rec(void *p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// Copies of source row position s (wrapped) into ring slot `slot`: the 8
// plane words of the lane's pair and its tile's stored-against reference.
template <typename T>
__device__ __forceinline__ void stage_row16(unsigned *ring, int lane, const Strip16 &a,
                                            const Coef<float> &k, int xa, int s, int slot,
                                            bool load) {
    if (load) {
        const int r = wave::wrap_row(s, a.ny);
        const T *base = (const T *)a.src;
        const T *p = base + (long long)r * a.nx + xa;
        unsigned *sl = ring + slot * W16_SLOT_WORDS;
#pragma unroll
        for (int i = 0; i < 8; ++i) cp_async4(sl + i * 32 + lane, p + (long long)i * a.plane);
        cp_async8w(sl + 8 * 32 + 2 * lane,
                   base + ref_at(k, (long long)r * k.tiles_x + (xa >> 3)));
    }
    wave::cp_commit();
}

// Sum over the 4 lanes of a tile (lanes b .. b + 3 hold its node pairs 0-1,
// 2-3, 4-5, 6-7) in the tree ((0 + 2) + (4 + 6)) + ((1 + 3) + (5 + 7)),
// formed in lane b (the pair sums of lanes b, b + 1 and of b + 2, b + 3 come
// down the warp; addition is commutative, so the order of the two operands
// does not change a bit).  Lanes other than b get partial sums; lanes of a
// tile the strip cuts (at its edges) get whatever the shuffles return: only
// whole tiles' sums are used.
__device__ __forceinline__ float tile_sum4_at_base(float2 v) {
    float2 t = f_add(v, make_float2(__shfl_down_sync(0xffffffffu, v.x, 1),
                                    __shfl_down_sync(0xffffffffu, v.y, 1)));
    t = f_add(t, make_float2(__shfl_down_sync(0xffffffffu, t.x, 2),
                             __shfl_down_sync(0xffffffffu, t.y, 2)));
    return f_add(t.x, t.y);
}

// The reference words of a tile from its nodes' pulled moments, as next_ref
// forms them, in lane b; `everyone`: also broadcast the sums from lane b to
// the tile's other lanes.
template <typename T>
__device__ __forceinline__ uint2 tile_next_ref(float2 rho, float2 mx, float2 my, int b,
                                               const Coef<float> &k, bool everyone) {
    float sr = tile_sum4_at_base(rho), sx = tile_sum4_at_base(mx), sy = tile_sum4_at_base(my);
    if (everyone) {
        sr = __shfl_sync(0xffffffffu, sr, b);
        sx = __shfl_sync(0xffffffffu, sx, b);
        sy = __shfl_sync(0xffffffffu, sy, b);
    }
    return next_ref<T>(sr, sx, sy, k, k.ref_gamma);
}

template <int K>
struct March16 {
    float2 w[K][3][8];      // windows of levels 0..K-1 (level 0: decoded source rows)
    uint2 enc;              // reference of the row level K stores next
    unsigned *ring;
};

// One march position s with s - s_lo = P (mod 3).
template <typename T, int K, int P, bool SEAM, bool SR, bool WALLS>
__device__ __forceinline__ void march_step16(March16<K> &m, const Strip16 &a,
                                             const Coef<float> &k, int s, int lane, int xa,
                                             int b, bool rec_lane, bool out_lane, bool seam_a,
                                             bool seam_b, bool walls, int y0, int y1, int s_lo,
                                             int s_load_hi) {
    const int rel = s - s_lo;
    stage_row16<T>(m.ring, lane, a, k, xa, s + W16_RING - 1, (rel + W16_RING - 1) % W16_RING,
                   s + W16_RING - 1 <= s_load_hi);
    wave::cp_wait<W16_RING - 1>();
    {   // level 0: row s decoded (stored value + reference population)
        const unsigned *sl = m.ring + (rel % W16_RING) * W16_SLOT_WORDS;
        const uint2 rw = *reinterpret_cast<const uint2 *>(sl + 8 * 32 + 2 * lane);
        float R[8];
        ref_pops(ref_of<T>(rw), k, R);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            m.w[0][P][i] = f_add(word_to_f2<T>(sl[i * 32 + lane]), make_float2(R[i], R[i]));
    }
    uint2 enc_next = m.enc;
#pragma unroll
    for (int l = 1; l <= K; ++l) {
        const int r = s - l;
        float2 d[8];
        wave::pull_level<SEAM, WALLS>(m.w[l - 1][mod3(P - l - 1)], m.w[l - 1][mod3(P - l)],
                               m.w[l - 1][mod3(P - l + 1)], k, seam_a, seam_b, walls, r, a.ny,
                               d);
        float2 rho, mx, my;
        moments_f32(d, rho, mx, my);
        relax_f32(d, rho, mx, my, k);
        // every lane of a tile stores against this reference: broadcast it
        if (l == K - 1) enc_next = tile_next_ref<T>(rho, mx, my, b, k, true);
        if (l < K) {
#pragma unroll
            for (int i = 0; i < 8; ++i) m.w[l][mod3(P - l)][i] = d[i];
        } else {
            // stored against the reference worked out at level K - 1 for
            // this row (one position ago), with the record of the tile
            const uint2 nxt = tile_next_ref<T>(rho, mx, my, b, k, false);   // lane b's record
            if (out_lane && r >= y0 && r < y1) {
                float Re[8];
                ref_pops(ref_of<T>(m.enc), k, Re);
                const long long node = (long long)r * a.nx + xa;
                T *o = (T *)a.dst + node;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    st_word(o + (long long)i * a.plane,
                            store_word<T, SR>(f_sub(d[i], make_float2(Re[i], Re[i])),
                                              (unsigned)(node >> 1), i));
                if (rec_lane)
                    st_rec((T *)a.dst + ref_at(k, (long long)r * k.tiles_x + (xa >> 3)),
                           make_uint4(m.enc.x, m.enc.y, nxt.x, nxt.y));
            }
        }
    }
    m.enc = enc_next;
}

// Halo of the 16-bit strips: 4 columns (>= K) for every K, so that the
// written columns, tx S .. tx S + 55 with S = 56, are whole tiles.
constexpr int H16 = 4;

// WALLS = false: y is periodic (the wall rule is left out of the code).
template <typename T, int K, bool SEAM, bool SR, bool WALLS>
__device__ __forceinline__ void run_strip16(const Strip16 &a, const Coef<float> &k, int tx,
                                            int sg, unsigned *warp_ring) {
    static_assert(K <= H16, "the halo must cover the steps");
    constexpr int H = H16;
    constexpr int S = wave::stride_of(H);
    static_assert(S % 8 == 0, "strips of whole tiles");
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const int x0 = tx * S - H;                       // column of lane 0's node a
    int xa = (x0 + 2 * lane) % nx;
    if (xa < 0) xa += nx;
    // position of the lane in its tile: columns x0 + 2 lane, x0 = tx S - H
    // with S a multiple of 8, so (x0 mod 8) / 2 = (8 - H) / 2
    const int o = ((8 - H) / 2 + lane) & 3;
    const int b = lane - o;                          // first lane of its tile
    const bool out_lane = lane >= H / 2 && lane < 32 - H / 2 && tx * S + 2 * (lane - H / 2) < nx;
    // the first lane of a whole tile inside the written columns writes the
    // tile's record (written columns start at tx S, a multiple of 8)
    const bool rec_lane = out_lane && o == 0;
    const bool grad = a.bc_x == BC_GRADIENT;
    const bool seam_a = grad && xa == 0;
    const bool seam_b = grad && xa + 2 == nx;
    const bool walls = WALLS && a.bc_y == BC_WALLS;
    const int y0 = sg * a.seg_rows;
    const int y1 = min(y0 + a.seg_rows, a.ny);
    const int s_lo = walls ? max(y0 - K, 0) : y0 - K;
    const int s_end = y1 - 1 + K;
    const int s_load_hi = walls ? min(y1 - 1 + K, a.ny - 1) : s_end;

    March16<K> m;
    m.ring = warp_ring;
    m.enc = make_uint2(0u, 0u);
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 8; ++i) m.w[l][j][i] = make_float2(0.f, 0.f);
    // every slot starts finite (zero words and references decode to 0)
    for (int j = lane; j < W16_RING * W16_SLOT_WORDS; j += 32) m.ring[j] = 0u;
    __syncwarp();
    for (int j = 0; j < W16_RING - 1; ++j)
        stage_row16<T>(m.ring, lane, a, k, xa, s_lo + j, j, s_lo + j <= s_load_hi);
    int s = s_lo;
    for (; s + 2 <= s_end; s += 3) {
        march_step16<T, K, 0, SEAM, SR, WALLS>(m, a, k, s, lane, xa, b, rec_lane, out_lane, seam_a,
                                        seam_b, walls, y0, y1, s_lo, s_load_hi);
        march_step16<T, K, 1, SEAM, SR, WALLS>(m, a, k, s + 1, lane, xa, b, rec_lane, out_lane, seam_a,
                                        seam_b, walls, y0, y1, s_lo, s_load_hi);
        march_step16<T, K, 2, SEAM, SR, WALLS>(m, a, k, s + 2, lane, xa, b, rec_lane, out_lane, seam_a,
                                        seam_b, walls, y0, y1, s_lo, s_load_hi);
    }
    if (s <= s_end)
        march_step16<T, K, 0, SEAM, SR, WALLS>(m, a, k, s, lane, xa, b, rec_lane, out_lane, seam_a,
                                        seam_b, walls, y0, y1, s_lo, s_load_hi);
    if (s + 1 <= s_end)
        march_step16<T, K, 1, SEAM, SR, WALLS>(m, a, k, s + 1, lane, xa, b, rec_lane, out_lane, seam_a,
                                        seam_b, walls, y0, y1, s_lo, s_load_hi);
    wave::cp_wait<0>();
}

// 12 warps per SM: the 4-step march fits 168 registers (with blocks of 4
// warps and a few bytes of spills this took FP16 at 8192^2 from 219 to 230
// GLUPS); fewer steps fit in fewer.
template <typename T, int K, bool SEAM, bool SR, bool WALLS>
__global__ void __launch_bounds__(W16_WARPS * 32, 12 / W16_WARPS)
step_wave16(const Strip16 a, const Coef<float> k, int tiles_x, long long items) {
    extern __shared__ unsigned w16_ring[];
    const long long item = (long long)blockIdx.x * W16_WARPS + (threadIdx.x >> 5);
    if (item >= items) return;                   // whole warps leave together
    run_strip16<T, K, SEAM, SR, WALLS>(a, k, int(item % tiles_x), int(item / tiles_x),
                                w16_ring + (threadIdx.x >> 5) * W16_RING * W16_SLOT_WORDS);
}

template <typename T, int K>
cudaError_t launch16_k(const Strip16 &a, const Coef<float> &k, cudaStream_t stream) {
    constexpr int S = wave::stride_of(H16);
    const int tiles_x = (a.nx + S - 1) / S;
    const long long segs = (a.ny + a.seg_rows - 1) / a.seg_rows;
    const long long items = (long long)tiles_x * segs;
    const long long blocks = (items + W16_WARPS - 1) / W16_WARPS;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool seam = a.bc_x == BC_GRADIENT, walls = a.bc_y == BC_WALLS;
    const unsigned g = (unsigned)blocks;
    constexpr int NT = W16_WARPS * 32;
    // stochastic rounding (opt-in) keeps the wall test at run time; the
    // nearest-rounding marches leave the wall rule out on periodic y
    if (seam && k.stochastic)
        step_wave16<T, K, true, true, true><<<g, NT, W16_SMEM, stream>>>(a, k, tiles_x, items);
    else if (k.stochastic)
        step_wave16<T, K, false, true, true><<<g, NT, W16_SMEM, stream>>>(a, k, tiles_x, items);
    else if (seam && walls)
        step_wave16<T, K, true, false, true><<<g, NT, W16_SMEM, stream>>>(a, k, tiles_x, items);
    else if (seam)
        step_wave16<T, K, true, false, false><<<g, NT, W16_SMEM, stream>>>(a, k, tiles_x, items);
    else if (walls)
        step_wave16<T, K, false, false, true><<<g, NT, W16_SMEM, stream>>>(a, k, tiles_x, items);
    else
        step_wave16<T, K, false, false, false><<<g, NT, W16_SMEM, stream>>>(a, k, tiles_x, items);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch16(int steps, const Strip16 &a, const Coef<float> &k, cudaStream_t stream) {
    switch (steps) {
        case 2: return launch16_k<T, 2>(a, k, stream);
        case 3: return launch16_k<T, 3>(a, k, stream);
        default: return launch16_k<T, 4>(a, k, stream);
    }
}

}  // namespace

cudaError_t launch_step_wave16(int precision, int steps, const void *src, void *dst, int nx,
                               int ny, int bc_x, int bc_y, const Coef<float> &k, int seg_rows,
                               cudaStream_t stream) {
    if (!wave_supported(precision, nx, ny, bc_x, bc_y) || !has_tile_refs(precision) ||
        steps < WAVE_MIN_STEPS || steps > WAVE16_MAX_STEPS || seg_rows < 1 || src == dst ||
        k.tile_shift != 3)
        return cudaErrorInvalidValue;
    Strip16 a;
    a.src = src;
    a.dst = dst;
    a.plane = (long long)nx * ny;
    a.nx = nx;
    a.ny = ny;
    a.bc_x = bc_x;
    a.bc_y = bc_y;
    a.seg_rows = seg_rows < ny ? seg_rows : ny;
    if (precision == PREC_FP16) return launch16<__half>(steps, a, k, stream);
    return launch16<__nv_bfloat16>(steps, a, k, stream);
}

}  // namespace plbm
