// 16-bit storage, two nodes at a time.
//
// A 16-byte vector of one population plane holds 8 consecutive nodes as 4
// words of two 16-bit values: word m holds nodes 2m (low half) and 2m + 1
// (high half).  The x shift of the pull (Eq. 13, left-hand side) is a funnel
// shift of those words by one 16-bit value, and each word converts to a
// float2 that is a node pair of one population, which the packed FP32 pair
// instructions collide at once (collide_f32<float2>: the same bits as the
// node-by-node collision).  The vector kernel and the staged kernel use this
// for 16-bit storage; inputs stay packed until their pair is collided, which
// keeps fewer values live than unpacking all 8 nodes first.
#pragma once

#include "lbm_device.cuh"

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

// A word's two 16-bit values as a float2 (low half -> x; exact) and back
// (x -> low half, rounded to nearest even, as Store<T>::put), in registers.
template <typename T> __device__ __forceinline__ float2 word_to_f2(unsigned w);
template <> __device__ __forceinline__ float2 word_to_f2<__half>(unsigned w) {
    float a, b;
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "cvt.f32.f16 %0, lo;\n\tcvt.f32.f16 %1, hi;\n\t}"
        : "=f"(a), "=f"(b)
        : "r"(w));
    return make_float2(a, b);
}
template <> __device__ __forceinline__ float2 word_to_f2<__nv_bfloat16>(unsigned w) {
    // a bfloat16 is the high half of the float with the same value
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <typename T> __device__ __forceinline__ unsigned f2_to_word(float2 v);
template <> __device__ __forceinline__ unsigned f2_to_word<__half>(float2 v) {
    unsigned r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(v.y), "f"(v.x));
    return r;
}
template <> __device__ __forceinline__ unsigned f2_to_word<__nv_bfloat16>(float2 v) {
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(v.y), "f"(v.x));
    return r;
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
// post-collision values of nodes 2m, 2m + 1 of population i.  hook(m, f)
// sees each pair's pulled state (after the walls, before the collision).
template <typename T, typename Hook = NoPairHook>
__device__ __forceinline__ void collide_words16(uint4 (&w)[8], const Coef<float> &k,
                                                const SeamAdd &seam, bool bottom, bool top,
                                                const Hook &hook = Hook()) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 f[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = word_to_f2<T>(word_of(w[i], m));
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
        collide_f32<float2>(f, k);
#pragma unroll
        for (int i = 0; i < 8; ++i) set_word(w[i], m, f2_to_word<T>(f[i]));
    }
}

}  // namespace plbm
