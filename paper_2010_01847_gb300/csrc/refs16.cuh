// 16-bit population storage relative to a local reference equilibrium.
//
// FP16 keeps 11 significant bits, BF16 8.  Stored as deviations from the
// rest equilibrium at one global reference energy, every population carries
// the whole local energy deviation w_i (e - e_ref), and the heat flux, a
// difference of populations (Eq. 54), keeps only what that cancellation
// leaves: where |q| is a fraction of |e - e_ref| its relative error per step
// is several storage units, and round-to-nearest errors of slowly varying
// fields add up step after step.  So the populations of each tile of
// 2^shift nodes of a row are stored relative to a reference equilibrium of
// the tile,
//     R_i = w_i rho_t + h_i c_i . j_t                  (the form of Eq. 15),
// with rho_t, j_t the tile means of the nodes' energy and post-collision
// first moment: what is stored is the non-equilibrium part of each node plus
// its departure from the tile mean, far smaller than the populations.
//
// The reference a tile's populations are stored against is the one its
// writer worked out in the step before (one step of lag): it is known before
// the collision, so a kernel collides, subtracts and stores each node (or
// node pair) in one pass, and it is as good as the current one (measured
// with the FP64 oracle in an emulation of the storage: FP16 errors after
// 5000 steps of the second-sound pulse 8e-5 with the lag, 2e-4 without).
//
// Layout: after the 8 population planes of nx ny values, a reference plane
// of 8 storage values per tile, tile t = y tiles_x + (x >> shift):
//   [0..2]  {rho_t, j_tx, j_ty} / 4 the tile's populations are stored against
//   [4..6]  {rho_t, j_tx, j_ty} / 4 worked out in this step (the next one's)
//   [3], [7] zero.
// (/4 keeps the FP16 values far below its largest finite number: |rho| is at
// most 1 / w_axis = 4.5 times the largest population.)  Tiles are 8 nodes
// (shift 3, the 16-byte vectors of the vector kernels) when nx is a multiple
// of 8, else single nodes (shift 0).  Every kernel forms each value with the
// same operations in the same order, the tile sums in the tree
// ((0 + 2) + (4 + 6)) + ((1 + 3) + (5 + 7)) over the tile's nodes, so all of
// them store the same bits.
#pragma once

#include "lbm_device.cuh"

namespace plbm {

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

// Stochastic rounding, an option of 16-bit storage (round-to-nearest is the
// default).  Round-to-nearest errors of slowly varying fields repeat step
// after step and add up; rounding up with probability equal to the dropped
// fraction makes each error zero on average, so they add like a random
// walk.  The random bits are a hash of the node pair (its global index),
// the plane and the two values' FP32 bits: deterministic, and the same in
// every kernel that stores the pair.  FP16 drops 13 bits of an FP32
// significand (normal range), BF16 16: those bits get a random number of
// that width added to the magnitude, then are cut off.
__device__ __forceinline__ unsigned sr_hash(unsigned pair, unsigned plane, unsigned a,
                                            unsigned b) {
    unsigned h = pair * 0x9E3779B1u ^ (plane + 1u) * 0x85EBCA77u ^ a ^ __funnelshift_l(b, b, 16);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}
// One value rounded stochastically with random bits r (below the kept
// significand), as the FP32 bit pattern of the result.
template <int DROP>
__device__ __forceinline__ unsigned sr_bits(float x, unsigned r) {
    const unsigned b = __float_as_uint(x);
    const unsigned mag = ((b & 0x7fffffffu) + (r & ((1u << DROP) - 1u))) & ~((1u << DROP) - 1u);
    return (b & 0x80000000u) | mag;
}
template <typename T> __device__ __forceinline__ unsigned f2_to_word_sr(float2 v, unsigned h);
template <> __device__ __forceinline__ unsigned f2_to_word_sr<__half>(float2 v, unsigned h) {
    // exact in FP16 after the cut (normal range), so the conversion keeps it
    return f2_to_word<__half>(make_float2(__uint_as_float(sr_bits<13>(v.x, h)),
                                          __uint_as_float(sr_bits<13>(v.y, h >> 16))));
}
template <> __device__ __forceinline__ unsigned f2_to_word_sr<__nv_bfloat16>(float2 v,
                                                                             unsigned h) {
    return (sr_bits<16>(v.x, h) >> 16) | (sr_bits<16>(v.y, h >> 16) & 0xffff0000u);
}
// A node pair (nodes 2 pair, 2 pair + 1 of the lattice, values v.x, v.y) of
// plane i as a stored word, rounded as SR says.
template <typename T, bool SR>
__device__ __forceinline__ unsigned store_word(float2 v, unsigned pair, int i) {
    if (SR)
        return f2_to_word_sr<T>(v, sr_hash(pair, (unsigned)i, __float_as_uint(v.x),
                                          __float_as_uint(v.y)));
    return f2_to_word<T>(v);
}

// One tile's reference {rho, jx, jy} / 4 in FP32.
struct Ref3 {
    float r, x, y;
};

// The two words {rho, jx}, {jy, 0} of a reference <-> its FP32 values.
template <typename T> __device__ __forceinline__ Ref3 ref_of(uint2 w) {
    const float2 a = word_to_f2<T>(w.x), b = word_to_f2<T>(w.y);
    return Ref3{a.x, a.y, b.x};
}
template <typename T> __device__ __forceinline__ uint2 ref_words(float r, float x, float y) {
    return make_uint2(f2_to_word<T>(make_float2(r, x)), f2_to_word<T>(make_float2(y, 0.f)));
}

// Element offset of tile t's 8 reference values in a state buffer.
__device__ __forceinline__ long long ref_at(const Coef<float> &k, long long tile) {
    return k.ref_off + 8 * tile;
}
// Tile of node (x, y).
__device__ __forceinline__ long long tile_of(const Coef<float> &k, int x, int y) {
    return (long long)y * k.tiles_x + (x >> k.tile_shift);
}

// The reference a tile's populations are stored against (read-only data of
// the step: through the non-coherent path).
template <typename T>
__device__ __forceinline__ uint2 ld_ref_stored(const T *buf, const Coef<float> &k, long long t) {
    return __ldg(reinterpret_cast<const uint2 *>(buf + ref_at(k, t)));
}
// Both references of a tile: .x/.y the stored-against one, .z/.w the next.
template <typename T>
__device__ __forceinline__ uint4 ld_ref_both(const T *buf, const Coef<float> &k, long long t) {
    return __ldg(reinterpret_cast<const uint4 *>(buf + ref_at(k, t)));
}
// Writes a tile's two references: `stored` (what its populations in this
// buffer are stored against) and `next`.
template <typename T>
__device__ __forceinline__ void st_ref(T *buf, const Coef<float> &k, long long t, uint2 stored,
                                       uint2 next) {
    *reinterpret_cast<uint4 *>(buf + ref_at(k, t)) = make_uint4(stored.x, stored.y, next.x, next.y);
}

// R_i of a reference (population i), in FP32: the coefficients of the
// collision times 4 (exact), t_i formed as in relax_f32.
template <int I>
__device__ __forceinline__ float ref_pop(const Ref3 &r, const Coef<float> &k) {
    constexpr bool axis = I < 4;
    const float w4 = axis ? k.rw_axis : k.rw_diag;
    const float h4 = axis ? k.rh_axis : k.rh_diag;
    // c_i . j: i = 0..7 -> x, y, -x, -y, x + y, -(x - y), -(x + y), x - y
    float t;
    if (I == 0 || I == 2) t = f_mul(h4, r.x);
    else if (I == 1 || I == 3) t = f_mul(h4, r.y);
    else if (I == 4 || I == 6) t = f_mul(h4, f_add(r.x, r.y));
    else t = f_mul(h4, f_sub(r.x, r.y));
    if (I == 2 || I == 3 || I == 5 || I == 6) t = -t;
    return f_fma(w4, r.r, t);
}
__device__ __forceinline__ float ref_pop_i(int i, const Ref3 &r, const Coef<float> &k) {
    switch (i) {
        case 0: return ref_pop<0>(r, k);
        case 1: return ref_pop<1>(r, k);
        case 2: return ref_pop<2>(r, k);
        case 3: return ref_pop<3>(r, k);
        case 4: return ref_pop<4>(r, k);
        case 5: return ref_pop<5>(r, k);
        case 6: return ref_pop<6>(r, k);
        default: return ref_pop<7>(r, k);
    }
}
// All 8 R_i of one reference.
__device__ __forceinline__ void ref_pops(const Ref3 &r, const Coef<float> &k, float (&R)[8]) {
    R[0] = ref_pop<0>(r, k);
    R[1] = ref_pop<1>(r, k);
    R[2] = ref_pop<2>(r, k);
    R[3] = ref_pop<3>(r, k);
    R[4] = ref_pop<4>(r, k);
    R[5] = ref_pop<5>(r, k);
    R[6] = ref_pop<6>(r, k);
    R[7] = ref_pop<7>(r, k);
}

// Tile sums in the fixed tree ((0 + 2) + (4 + 6)) + ((1 + 3) + (5 + 7)):
// of 8 values of one thread, of 4 node pairs (pair m = nodes 2m, 2m + 1), and
// across the 8 lanes of an aligned lane group (every lane of the warp calls
// it; each lane of the group gets the sum).
__device__ __forceinline__ float tile_tree8(const float (&v)[8]) {
    return f_add(f_add(f_add(v[0], v[2]), f_add(v[4], v[6])),
                 f_add(f_add(v[1], v[3]), f_add(v[5], v[7])));
}
__device__ __forceinline__ float tile_tree_pairs(float2 p01, float2 p23) {
    const float2 q = f_add(p01, p23);
    return f_add(q.x, q.y);
}
__device__ __forceinline__ float tile_tree_lanes(float v) {
    v = f_add(v, __shfl_xor_sync(0xffffffffu, v, 2));
    v = f_add(v, __shfl_xor_sync(0xffffffffu, v, 4));
    return f_add(v, __shfl_xor_sync(0xffffffffu, v, 1));
}

// The next reference of a tile from its sums of rho and m (pulled moments,
// moments_f32): {rho, gamma m} / (4 nodes-per-tile), rounded to the storage
// type.  `j_factor` is k.ref_gamma after a collision (the post-collision
// first moment is gamma m), k.ref_rho for a state before collision.
template <typename T>
__device__ __forceinline__ uint2 next_ref(float s_rho, float s_mx, float s_my,
                                          const Coef<float> &k, float j_factor) {
    return ref_words<T>(f_mul(s_rho, k.ref_rho), f_mul(s_mx, j_factor), f_mul(s_my, j_factor));
}

// pull_node_with reading global post-collision planes (the scalar step
// kernels and the scalar read-outs); with 16-bit storage each value gets the
// reference population of the tile it is pulled from.
template <typename T>
__device__ __forceinline__ void pull_node(const T *__restrict__ src, long long plane,
                                          int nx, int ny, int x, int y, int bc_x,
                                          int bc_y, const Coef<typename Store<T>::C> &k,
                                          typename Store<T>::C (&d)[8]) {
    using C = typename Store<T>::C;
    pull_node_with(
        [&](int i, int sx, int sy) -> C {
            const C v = Store<T>::load(src[(long long)i * plane + (long long)sy * nx + sx]);
            if constexpr (sizeof(T) == 2)
                return f_add(v, ref_pop_i(i, ref_of<T>(ld_ref_stored(src, k, tile_of(k, sx, sy))),
                                          k));
            else
                return v;
        },
        nx, ny, x, y, bc_x, bc_y, k, d);
}

// The references a vector thread needs (16-bit storage, tiles of 8 nodes =
// its 16-byte vectors: tile column xv of row y).  Rd[i]: the reference
// population of the tile it pulls plane i from (row y - c_iy, column xv);
// for a lane at a warp edge or a row end (need_left / need_right) also
// Rx[i], the same for the neighbouring tile its node 0 (c_x = +1) or node 7
// (c_x = -1) is pulled from (other lanes take theirs from the adjacent
// lane); enc: the reference its own tile is stored against next.  Rows and
// columns wrap, so every load stays inside the lattice.  The loads
// (vector_ref_loads) are issued apart from the arithmetic (vector_ref_pops)
// so that they can fly together with the population loads.
struct VecRefWords {
    uint4 own;                  // row y: stored-against and next
    uint2 up, dn;               // rows y - 1, y + 1: stored-against
    uint2 l0, lu, ld, r0, ru, rd;   // neighbouring tiles (edge lanes only)
};
template <typename T>
__device__ __forceinline__ VecRefWords vector_ref_loads(const T *src, const Coef<float> &k,
                                                        int ny, int y, int xv, bool need_left,
                                                        bool need_right) {
    const int tpr = k.tiles_x;
    const long long ym = y == 0 ? ny - 1 : y - 1, y0 = y, yp = y + 1 == ny ? 0 : y + 1;
    VecRefWords r;
    r.own = ld_ref_both(src, k, y0 * tpr + xv);
    r.up = ld_ref_stored(src, k, ym * tpr + xv);
    r.dn = ld_ref_stored(src, k, yp * tpr + xv);
    r.l0 = r.lu = r.ld = r.r0 = r.ru = r.rd = make_uint2(0u, 0u);
    if (need_left) {
        const int xl = xv == 0 ? tpr - 1 : xv - 1;
        r.l0 = ld_ref_stored(src, k, y0 * tpr + xl);
        r.lu = ld_ref_stored(src, k, ym * tpr + xl);
        r.ld = ld_ref_stored(src, k, yp * tpr + xl);
    }
    if (need_right) {
        const int xr = xv + 1 == tpr ? 0 : xv + 1;
        r.r0 = ld_ref_stored(src, k, y0 * tpr + xr);
        r.ru = ld_ref_stored(src, k, ym * tpr + xr);
        r.rd = ld_ref_stored(src, k, yp * tpr + xr);
    }
    return r;
}
template <typename T>
__device__ __forceinline__ void vector_ref_pops(const VecRefWords &r, const Coef<float> &k,
                                                bool need_left, bool need_right, float (&Rd)[8],
                                                float (&Rx)[8], uint2 &enc) {
    enc = make_uint2(r.own.z, r.own.w);
    // plane i is pulled from row y - c_iy: c_y = 0 -> y, +1 -> y - 1, -1 -> y + 1
    const Ref3 a0 = ref_of<T>(make_uint2(r.own.x, r.own.y)), au = ref_of<T>(r.up),
               ad = ref_of<T>(r.dn);
    Rd[0] = ref_pop<0>(a0, k);
    Rd[2] = ref_pop<2>(a0, k);
    Rd[1] = ref_pop<1>(au, k);
    Rd[4] = ref_pop<4>(au, k);
    Rd[5] = ref_pop<5>(au, k);
    Rd[3] = ref_pop<3>(ad, k);
    Rd[6] = ref_pop<6>(ad, k);
    Rd[7] = ref_pop<7>(ad, k);
#pragma unroll
    for (int i = 0; i < 8; ++i) Rx[i] = 0.f;
    if (need_left) {          // c_x = +1 planes: 0 (row y), 4 (y - 1), 7 (y + 1)
        Rx[0] = ref_pop<0>(ref_of<T>(r.l0), k);
        Rx[4] = ref_pop<4>(ref_of<T>(r.lu), k);
        Rx[7] = ref_pop<7>(ref_of<T>(r.ld), k);
    }
    if (need_right) {         // c_x = -1 planes: 2 (row y), 5 (y - 1), 6 (y + 1)
        Rx[2] = ref_pop<2>(ref_of<T>(r.r0), k);
        Rx[5] = ref_pop<5>(ref_of<T>(r.ru), k);
        Rx[6] = ref_pop<6>(ref_of<T>(r.rd), k);
    }
}
// Rx of the lanes inside a warp: the neighbouring tile's reference
// population is the adjacent lane's Rd (same rows, next tile column).  Every
// lane calls it; lanes at a warp edge or a row end keep the Rx they loaded.
__device__ __forceinline__ void pull_edge_refs(const float (&Rd)[8], float (&Rx)[8],
                                               bool need_left, bool need_right) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (cx_of(i) > 0) {
            const float v = __shfl_up_sync(0xffffffffu, Rd[i], 1);
            if (!need_left) Rx[i] = v;
        } else if (cx_of(i) < 0) {
            const float v = __shfl_down_sync(0xffffffffu, Rd[i], 1);
            if (!need_right) Rx[i] = v;
        }
    }
}

template <typename T>
__device__ __forceinline__ void vector_refs(const T *src, const Coef<float> &k, int ny, int y,
                                            int xv, bool need_left, bool need_right,
                                            float (&Rd)[8], float (&Rx)[8], uint2 &enc) {
    vector_ref_pops<T>(vector_ref_loads<T>(src, k, ny, y, xv, need_left, need_right), k,
                       need_left, need_right, Rd, Rx, enc);
}

}  // namespace plbm
