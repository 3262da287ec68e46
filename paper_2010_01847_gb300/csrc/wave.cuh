// The strip march of the multi-step stream-collide kernel (shared by the
// single-lattice kernel in wave.cu and the batched one in batch.cu).
//
// One warp owns a strip of 64 columns (two adjacent nodes per lane, one
// float2 per plane) and a segment of rows, and marches up the rows.  At
// march position s it brings in the post-collision row s of the source
// planes (level 0) and advances every level l = 1..K by one row: level l
// computes row s - l from rows s - l - 1, s - l, s - l + 1 of level l - 1,
// which the warp holds in registers (each level keeps a window of three rows,
// slot = row position mod 3; only the planes a later pull reads stay live).
// The pull takes the c_y neighbour from the window row above or below and
// the c_x neighbour from the lane's other node or, across lanes, by a warp
// shuffle; then the seam jump (Eqs. 59-60), the diffuse walls (Eq. 58) and
// the collision (collide_f32 on the node pair: the same operations, in the
// same order, as every other FP32 kernel, so the result is bit-identical to
// K single steps).  Level K rows are written to the destination planes.
//
// The source rows come through a ring of RING rows per warp in shared
// memory, filled by cp.async copies issued RING - 1 positions ahead, so the
// loads of later rows are in flight while the levels compute.
//
// A strip's outer columns depend on columns outside it: after l levels the
// l outermost columns on each side are wrong, so the strip overlaps its
// neighbours by a halo of H >= K columns each side (even, so that pairs stay
// 8-byte aligned) and writes only its 64 - 2H middle columns.  Likewise a
// segment of rows [y0, y1) starts its march K rows early and ends K rows
// late (periodic y), or at the walls, where no rows lie beyond (the wall
// rule of Eq. 58 replaces every population that would come from beyond
// them).
//
// Bytes per site update: one read and one write of the 8 planes per K steps,
// (32 + 32) / K B plus the halo rows re-read by adjacent segments (2K / rows
// of the reads); the halo columns are read by two strips at nearly the same
// time and come from L2.  The FP32 march requires nx even, x periodic (with
// or without the seam gradient) and y periodic or walled; no sides.  The
// 16-bit march (wave16.cu) reuses pull_level and the ring helpers.
#pragma once

#include "lbm_device.cuh"

namespace plbm {
namespace wave {

constexpr int RING = 4;                    // source rows staged per warp (3 in flight ahead)
constexpr int RING_ELEMS = RING * 8 * 32;  // float2 of one warp's ring

// the smallest halo for K steps (columns per side, even: 8-byte pairs) and
// the columns a strip with halo H writes
__host__ __device__ constexpr int halo(int K) { return (K + 1) & ~1; }
__host__ __device__ constexpr int stride_of(int H) { return 64 - 2 * H; }

// One lattice as a strip march sees it: source and destination planes
// (post-collision, element offset 0 = plane 0, node 0) and segment rows.
struct Strip {
    const float *src;
    float *dst;
    long long plane;
    int nx, ny, bc_x, bc_y;
    int seg_rows;
};

__device__ __forceinline__ void st_pair(float *p, float2 v) {
    asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

constexpr int mod3(int v) { return ((v % 3) + 3) % 3; }

// The state of one strip's march: K windows of 3 rows x 8 planes (levels
// 0..K-1) in registers; the source rows come through the warp's ring of
// RING rows in shared memory (slot = row position mod RING; each lane
// copies and reads only its own pair of each plane).
template <int K>
struct March {
    float2 w[K][3][8];
    float2 *ring;        // this lane's element of slot 0, plane 0
};

__device__ __forceinline__ void cp_async8(float2 *dst, const float *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Row position s wrapped into [0, ny): one compare in the march's middle, a
// subtraction or addition of ny within K rows of its ends, and the remainder
// only for lattices fewer rows high than the march runs past them (s is the
// same in every lane).
__device__ __forceinline__ int wrap_row(int s, int ny) {
    if (s >= 0 && s < ny) return s;
    if (s >= ny && s < 2 * ny) return s - ny;
    if (s < 0 && s >= -ny) return s + ny;
    const int r = s % ny;
    return r < 0 ? r + ny : r;
}

// Issues the copies of source row position s (wrapped into [0, ny)) into
// its ring slot, as one commit group (an empty group past the last row, so
// the group count per position stays one).
__device__ __forceinline__ void stage_row(float2 *ring, const Strip &a, int xa, int s, int slot,
                                          bool load) {
    if (load) {
        const int r = wrap_row(s, a.ny);
        const float *p = a.src + (long long)r * a.nx + xa;
#pragma unroll
        for (int i = 0; i < 8; ++i) cp_async8(ring + (slot * 8 + i) * 32, p + (long long)i * a.plane);
    }
    cp_commit();
}

// The pull of one row of a level from rows r - 1, r, r + 1 of the level
// below (Eq. 13 left-hand side on the lane's node pair: c_y from the row
// below or above, c_x from the lane's other node or the neighbouring lane),
// the seam jump (Eqs. 59-60) and the walls (Eq. 58).  Every lane calls it.
// WALLS = false: the lattice has no walls (the wall rule is not compiled).
template <bool SEAM, bool WALLS = true>
__device__ __forceinline__ void pull_level(const float2 (&below)[8], const float2 (&here)[8],
                                           const float2 (&above)[8], const Coef<float> &k,
                                           bool seam_a, bool seam_b, bool walls, int r, int ny,
                                           float2 (&d)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        const float2 v = cy > 0 ? below[i] : (cy < 0 ? above[i] : here[i]);
        const float jw = i < 4 ? k.jump_axis : k.jump_diag;
        if (cx > 0) {        // node a from the left lane's node b, node b from node a
            float left = __shfl_up_sync(0xffffffffu, v.y, 1);
            if (SEAM && seam_a) left = left + jw;            // Eq. 59
            d[i] = make_float2(left, v.x);
        } else if (cx < 0) { // node b from the right lane's node a, node a from node b
            float right = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (SEAM && seam_b) right = right - jw;          // Eq. 60
            d[i] = make_float2(v.y, right);
        } else {
            d[i] = v;
        }
    }
    if (WALLS && walls) {
        if (r == 0) wall_bottom(d, k);
        if (r == ny - 1) wall_top(d, k);
    }
}

// One march position s with s - s_lo = P (mod 3).  SEAM: some lane of the
// warp pulls across the seam of a gradient lattice (else no jump is added).
template <int K, int P, bool SEAM, bool WALLS>
__device__ __forceinline__ void march_step(March<K> &m, const Strip &a, const Coef<float> &k,
                                           int s, int xa, bool out_lane, bool seam_a,
                                           bool seam_b, bool walls, int y0, int y1,
                                           int s_lo, int s_load_hi) {
    // stage row s + RING - 1, then wait for row s (RING - 1 groups may stay
    // in flight) and take it as level 0 (past the top wall a stale row,
    // which only wall unknowns ever read)
    const int rel = s - s_lo;
    stage_row(m.ring, a, xa, s + RING - 1, (rel + RING - 1) % RING,
              s + RING - 1 <= s_load_hi);
    cp_wait<RING - 1>();
    const int slot = rel % RING;
#pragma unroll
    for (int i = 0; i < 8; ++i) m.w[0][P][i] = m.ring[(slot * 8 + i) * 32];

    // Every level advances at every position, also on rows it does not need
    // (before the segment's first valid rows, or beyond a wall: finite
    // values no valid row reads), so each window slot is overwritten every
    // third position and only the planes still to be pulled stay live.
#pragma unroll
    for (int l = 1; l <= K; ++l) {
        const int r = s - l;
        const float2(&below)[8] = m.w[l - 1][mod3(P - l - 1)];   // row r - 1
        const float2(&here)[8] = m.w[l - 1][mod3(P - l)];        // row r
        const float2(&above)[8] = m.w[l - 1][mod3(P - l + 1)];   // row r + 1
        float2 d[8];
        pull_level<SEAM, WALLS>(below, here, above, k, seam_a, seam_b, walls, r, a.ny, d);
        collide_f32<float2>(d, k);
        if (l < K) {
#pragma unroll
            for (int i = 0; i < 8; ++i) m.w[l][mod3(P - l)][i] = d[i];
        } else if (out_lane && r >= y0 && r < y1) {
            float *p = a.dst + (long long)r * a.nx + xa;
#pragma unroll
            for (int i = 0; i < 8; ++i) st_pair(p + (long long)i * a.plane, d[i]);
        }
    }
}

// The march of strip tx (columns tx S - H .. tx S + 63 - H, wrapped,
// S = 64 - 2H), segment sg (rows sg seg_rows ..) of lattice a: K steps from
// a.src into a.dst.  H: the halo, even and >= K (a batch keeps one strip
// layout for launches of fewer steps).  SEAM: the lattice has the seam
// gradient (without it no jump is added: fewer instructions per level).
// WALLS = false: y is periodic (the wall rule is left out of the code).
// Every lane of the warp calls it (shuffles); warp_ring is the warp's
// RING_ELEMS float2 of shared memory.
template <int K, bool SEAM, bool WALLS = true>
__device__ __forceinline__ void run_strip(const Strip &a, const Coef<float> &k, int tx, int sg,
                                          int H, float2 *warp_ring) {
    const int S = stride_of(H);
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    int xa = (tx * S - H + 2 * lane) % nx;               // the lane's nodes: xa, xa + 1
    if (xa < 0) xa += nx;
    const bool out_lane = lane >= H / 2 && lane < 32 - H / 2 && tx * S + 2 * (lane - H / 2) < nx;
    const bool grad = a.bc_x == BC_GRADIENT;
    const bool seam_a = grad && xa == 0;          // node a pulls c_x = +1 across the seam
    const bool seam_b = grad && xa + 2 == nx;     // node b pulls c_x = -1 across it
    const bool walls = WALLS && a.bc_y == BC_WALLS;
    const int y0 = sg * a.seg_rows;
    const int y1 = min(y0 + a.seg_rows, a.ny);
    const int s_lo = walls ? max(y0 - K, 0) : y0 - K;
    const int s_end = y1 - 1 + K;
    const int s_load_hi = walls ? min(y1 - 1 + K, a.ny - 1) : s_end;

    March<K> m;
    m.ring = warp_ring + lane;
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 8; ++i) m.w[l][j][i] = make_float2(0.f, 0.f);
    // every slot starts finite (a wall lattice may read a slot it never
    // filled, as wall unknowns only); then rows s_lo .. s_lo + RING - 2
#pragma unroll
    for (int j = 0; j < RING * 8; ++j) m.ring[j * 32] = make_float2(0.f, 0.f);
    __syncwarp();
    for (int j = 0; j < RING - 1; ++j)
        stage_row(m.ring, a, xa, s_lo + j, j, s_lo + j <= s_load_hi);
    // whole rounds of three positions, then the remainder: no round skips
    // a position, so no slot keeps a value past its third position
    int s = s_lo;
    for (; s + 2 <= s_end; s += 3) {
        march_step<K, 0, SEAM, WALLS>(m, a, k, s, xa, out_lane, seam_a, seam_b, walls, y0, y1, s_lo, s_load_hi);
        march_step<K, 1, SEAM, WALLS>(m, a, k, s + 1, xa, out_lane, seam_a, seam_b, walls, y0, y1,
                         s_lo, s_load_hi);
        march_step<K, 2, SEAM, WALLS>(m, a, k, s + 2, xa, out_lane, seam_a, seam_b, walls, y0, y1,
                         s_lo, s_load_hi);
    }
    if (s <= s_end)
        march_step<K, 0, SEAM, WALLS>(m, a, k, s, xa, out_lane, seam_a, seam_b, walls, y0, y1, s_lo, s_load_hi);
    if (s + 1 <= s_end)
        march_step<K, 1, SEAM, WALLS>(m, a, k, s + 1, xa, out_lane, seam_a, seam_b, walls, y0, y1,
                         s_lo, s_load_hi);
    cp_wait<0>();          // nothing of this march left in flight
}

}  // namespace wave
}  // namespace plbm
