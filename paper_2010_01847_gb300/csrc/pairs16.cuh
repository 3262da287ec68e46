// 16-bit storage, two nodes at a time.
//
// A 16-byte vector of one population plane holds 8 consecutive nodes as 4
// words of two 16-bit values: word m holds nodes 2m (low half) and 2m + 1
// (high half).  The x shift of the pull (Eq. 13, left-hand side) is a funnel
// shift of those words by one 16-bit value, and each word converts to a
// float2 that is a node pair of one population, which the packed FP32 pair
// instructions collide at once (collide_f32<float2>: the same bits as the
// node-by-node collision).  The vector kernels use this for 16-bit storage;
// inputs stay packed until their pair is collided, which keeps fewer values
// live than unpacking all 8 nodes first.
#pragma once

#include "refs16.cuh"

namespace plbm {

// (high half of lo_src) | (low half of hi_src) << 16
__device__ __forceinline__ unsigned funnel16(unsigned lo_src, unsigned hi_src) {
    return __byte_perm(lo_src, hi_src, 0x5432);
}

// Node j takes node j - 1 (c_x = +1): `nb` holds the node left of node 0 in
// its high half.
__device__ __forceinline__ uint4 shift_from_left(uint4 v, unsigned nb) {
    return make_uint4(funnel16(nb, v.x), funnel16(v.x, v.y), funnel16(v.y, v.z),
                      funnel16(v.z, v.w));
}
// Node j takes node j + 1 (c_x = -1): `nb` holds the node right of node 7
// in its low half.
__device__ __forceinline__ uint4 shift_from_right(uint4 v, unsigned nb) {
    return make_uint4(funnel16(v.x, v.y), funnel16(v.y, v.z), funnel16(v.z, v.w),
                      funnel16(v.w, nb));
}

__device__ __forceinline__ unsigned word_of(const uint4 &v, int m) {
    return m == 0 ? v.x : m == 1 ? v.y : m == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_word(uint4 &v, int m, unsigned r) {
    if (m == 0) v.x = r;
    else if (m == 1) v.y = r;
    else if (m == 2) v.z = r;
    else v.w = r;
}

// Seam jumps (Eqs. 59-60) on the edge nodes of a thread's 8, in FP32 after
// conversion, as the node-by-node kernels add them: with `left`, node 0 of
// every c_x = +1 population gets + (the jump if `left_jump`, else 0); with
// `right`, node 7 of every c_x = -1 population gets - (the jump if
// `right_jump`, else 0).  The jump is s w_i delta_e (axis or diagonal).
struct SeamAdd {
    bool left, left_jump, right, right_jump;
};

// Does nothing with a node pair's pulled state (the plain step).
struct NoPairHook {
    __device__ __forceinline__ void operator()(int, const float2 (&)[8]) const {}
};

// Walls (Eq. 58 on the bottom / top row), collision, and repacking of the 8
// nodes held in w (after the shift), in place: word m of w[i] becomes the
// post-collision values of nodes 2m, 2m + 1 of population i.  With storage
// relative to tile references (refs16.cuh) every pulled value of plane i
// first gets Rd[i] added (the reference population of the tile it was
// pulled from), except the node shifted in from the neighbouring tile of a
// c_x = +1 (node 0) or c_x = -1 (node 7) plane, which gets Rx[i]; the
// post-collision values are stored less Re[i] (the reference of this tile
// for the next step's readers), and the tile's sums of rho, m_x, m_y
// (moments_f32, tree order of tile_tree_pairs) come back in sums.
// hook(m, f) sees each pair's pulled state (after the walls, before the
// collision).  SR: stochastic rounding of the stored values (refs16.cuh),
// pair0 the global index of the thread's first node pair.
template <typename T, bool SR = false, typename Hook = NoPairHook>
__device__ __forceinline__ void collide_words16(uint4 (&w)[8], const Coef<float> &k,
                                                const SeamAdd &seam, bool bottom, bool top,
                                                const float (&Rd)[8], const float (&Rx)[8],
                                                const float (&Re)[8], float (&sums)[3],
                                                unsigned pair0 = 0u, const Hook &hook = Hook()) {
    float2 r01, x01, y01, r23, x23, y23;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 f[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float2 R = make_float2(Rd[i], Rd[i]);
            if (m == 0 && cx_of(i) > 0) R.x = Rx[i];
            if (m == 3 && cx_of(i) < 0) R.y = Rx[i];
            f[i] = f_add(word_to_f2<T>(word_of(w[i], m)), R);
        }
        if (m == 0 && seam.left) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (cx_of(i) > 0)
                    f[i].x = f_add(f[i].x, seam.left_jump ? (i < 4 ? k.jump_axis : k.jump_diag)
                                                          : 0.f);
        }
        if (m == 3 && seam.right) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (cx_of(i) < 0)
                    f[i].y = f_sub(f[i].y, seam.right_jump ? (i < 4 ? k.jump_axis : k.jump_diag)
                                                           : 0.f);
        }
        if (bottom) wall_bottom(f, k);
        if (top) wall_top(f, k);
        hook(m, f);
        float2 rho, mx, my;
        moments_f32(f, rho, mx, my);
        if (m == 0) { r01 = rho; x01 = mx; y01 = my; }
        if (m == 1) { r01 = f_add(r01, rho); x01 = f_add(x01, mx); y01 = f_add(y01, my); }
        if (m == 2) { r23 = rho; x23 = mx; y23 = my; }
        if (m == 3) { r23 = f_add(r23, rho); x23 = f_add(x23, mx); y23 = f_add(y23, my); }
        relax_f32(f, rho, mx, my, k);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            set_word(w[i], m,
                     store_word<T, SR>(f_sub(f[i], make_float2(Re[i], Re[i])), pair0 + m, i));
    }
    sums[0] = tile_tree_pairs(r01, r23);
    sums[1] = tile_tree_pairs(x01, x23);
    sums[2] = tile_tree_pairs(y01, y23);
}

}  // namespace plbm
