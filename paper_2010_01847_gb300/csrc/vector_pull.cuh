// Vectorised pull shared by the vector stream-collide kernel and the
// vectorised read-out kernels: each thread owns V = 16/sizeof(T) consecutive
// nodes of one row and moves every plane with one aligned 16-byte load.  The
// x-shifted populations (c_x = +-1) take their out-of-vector neighbour from
// the adjacent lane by a warp shuffle; the first/last lane of a warp, and
// rows' ends, load that one element directly (wrapping at the seam, with the
// jump of Eqs. 59-60).  Requires nx % V == 0.  Threads are laid out
// row-major over the lattice, so a warp may straddle two rows; the row test
// handles that.  Every lane of a warp must call it (shuffles).
#pragma once

#include "refs16.cuh"

namespace plbm {

// 16-byte vector packing of V = 16/sizeof(T) consecutive plane elements.
template <typename T> struct Pack;
template <> struct Pack<float> {
    static constexpr int V = 4;
    __device__ static void unpack(uint4 r, float (&o)[4]) {
        o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
        o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
    }
    __device__ static uint4 pack(const float (&o)[4]) {
        return make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]),
                          __float_as_uint(o[2]), __float_as_uint(o[3]));
    }
};
template <> struct Pack<double> {
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
template <> struct Pack<__half> {
    static constexpr int V = 8;
    __device__ static float2 w2f(unsigned w) {
        __half2 h = *reinterpret_cast<__half2 *>(&w);
        return __half22float2(h);
    }
    __device__ static unsigned f2w(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<unsigned *>(&h);
    }
    __device__ static void unpack(uint4 r, float (&o)[8]) {
        float2 a = w2f(r.x), b = w2f(r.y), c = w2f(r.z), d = w2f(r.w);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
    }
    __device__ static uint4 pack(const float (&o)[8]) {
        return make_uint4(f2w(o[0], o[1]), f2w(o[2], o[3]), f2w(o[4], o[5]), f2w(o[6], o[7]));
    }
};
template <> struct Pack<__nv_bfloat16> {
    static constexpr int V = 8;
    __device__ static float2 w2f(unsigned w) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
        return __bfloat1622float2(h);
    }
    __device__ static unsigned f2w(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<unsigned *>(&h);
    }
    __device__ static void unpack(uint4 r, float (&o)[8]) {
        float2 a = w2f(r.x), b = w2f(r.y), c = w2f(r.z), d = w2f(r.w);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
    }
    __device__ static uint4 pack(const float (&o)[8]) {
        return make_uint4(f2w(o[0], o[1]), f2w(o[2], o[3]), f2w(o[4], o[5]), f2w(o[6], o[7]));
    }
};

__device__ __forceinline__ uint4 ld_stream(const void *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ void st_stream(void *p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}


// V consecutive values of the compute type C (16 or 32 bytes, 16-byte
// aligned) as 16-byte vector accesses.
template <typename C, int V>
__device__ __forceinline__ void load_cvec(const C *__restrict__ p, C (&v)[V]) {
    static_assert((V * sizeof(C)) % 16 == 0, "whole 16-byte chunks");
#pragma unroll
    for (int c = 0; c < (int)(V * sizeof(C) / 16); ++c)
        reinterpret_cast<uint4 *>(v)[c] = reinterpret_cast<const uint4 *>(p)[c];
}
template <typename C, int V>
__device__ __forceinline__ void store_cvec(C *__restrict__ p, const C (&v)[V]) {
#pragma unroll
    for (int c = 0; c < (int)(V * sizeof(C) / 16); ++c)
        reinterpret_cast<uint4 *>(p)[c] = reinterpret_cast<const uint4 *>(v)[c];
}

// Residual terms of a thread's V pulled nodes (walls already applied),
// history planes read and written as 16-byte vectors.
template <typename C, int V>
__device__ __forceinline__ void residual_vec(const C (&n)[V][8], const Coef<C> &k, C inv_s,
                                             C *__restrict__ prev, long long plane,
                                             long long out, bool have_prev, C (&loc)[5]) {
    C h[3][V];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (have_prev) {
            load_cvec<C, V>(prev + q * plane + out, h[q]);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) h[q][j] = C(0);
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) residual_terms(n[j], k, inv_s, h[0][j], h[1][j], h[2][j],
                                               have_prev, loc);
#pragma unroll
    for (int q = 0; q < 3; ++q) store_cvec<C, V>(prev + q * plane + out, h[q]);
}

// Position of a thread's vector and the rows it touches.
struct VecPos {
    int y, xv, x0;
    bool active, bottom, top;
};

// Pulls the populations arriving at the thread's V nodes (Eq. 13 left-hand
// side, seam jump); wall unknowns are left at 0 for the caller's Eq. 58.
// With SIDES, directions created with BC_SIDES are not periodic either:
// populations that would come from beyond a side are left at 0 for the
// caller's apply_sides (bottom/top then also flag the rows of y sides).
// 16-bit storage: the values are stored relative to tile references
// (refs16.cuh); each is pulled with its tile's reference population added
// (before the shift, so the neighbour's value arrives complete), and *enc
// (if given) receives the reference this thread's tile is stored against
// next.
template <typename T, bool SIDES = false>
__device__ __forceinline__ VecPos vector_pull(const T *__restrict__ src, int nx, int ny,
                                              long long plane, int bc_x, int bc_y,
                                              const Coef<typename Store<T>::C> &k, long long t,
                                              typename Store<T>::C (&d)[8][Pack<T>::V],
                                              uint2 *enc = nullptr) {
    using C = typename Store<T>::C;
    constexpr int V = Pack<T>::V;
    const int tpr = nx / V;
    const long long total = (long long)tpr * ny;
    const bool active = t < total;
    const int y = active ? int(t / tpr) : 0;
    const int xv = active ? int(t - (long long)y * tpr) : 0;
    const int x0 = xv * V;
    const int lane = threadIdx.x & 31;
    const bool walls = bc_y == BC_WALLS || (SIDES && bc_y == BC_SIDES);
    const bool bottom = walls && y == 0;
    const bool top = walls && y == ny - 1;
    const bool open_x = SIDES && bc_x == BC_SIDES;
    const bool left_side = open_x && x0 == 0;          // no node beyond x = 0
    const bool right_side = open_x && x0 + V == nx;    // none beyond x = nx - 1

    // every load is issued before any is used: the 16-byte vectors and, for
    // the lanes at a warp edge or a row end, the one neighbouring element of
    // each x-shifted plane (so a warp waits for one memory round trip)
    const bool need_left = (lane == 0 || xv == 0) && active;
    const bool need_right = (lane == 31 || xv + 1 == tpr) && active;
    const int sx_left = x0 == 0 ? nx - 1 : x0 - 1;
    const int sx_right = x0 + V >= nx ? x0 + V - nx : x0 + V;
    VecRefWords rw{};
    if constexpr (sizeof(T) == 2) rw = vector_ref_loads<T>(src, k, ny, y, xv, need_left, need_right);
    C edge[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        int sy = y - cy;
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        const long long row = (long long)i * plane + (long long)sy * nx;
        const bool unknown = (cy > 0 && bottom) || (cy < 0 && top);
        if (active && !unknown) {
            Pack<T>::unpack(ld_stream(src + row + x0), d[i]);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) d[i][j] = C(0);
        }
        edge[i] = C(0);
        if (cx > 0 && need_left && !unknown && !left_side)
            edge[i] = Store<T>::load(src[row + sx_left]);
        if (cx < 0 && need_right && !unknown && !right_side)
            edge[i] = Store<T>::load(src[row + sx_right]);
    }

    if constexpr (sizeof(T) == 2) {
        float Rd[8], Rx[8];
        uint2 e2;
        vector_ref_pops<T>(rw, k, need_left, need_right, Rd, Rx, e2);
        if (enc) *enc = e2;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = 0; j < V; ++j) d[i][j] = f_add(d[i][j], Rd[i]);
            if (cx_of(i) != 0) edge[i] = f_add(edge[i], Rx[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i);
        if (cx == 0) continue;
        const C jw = (i < 4) ? k.jump_axis : k.jump_diag;
        if (cx > 0) {
            C left = __shfl_up_sync(0xffffffffu, d[i][V - 1], 1);
            if (need_left) {
                // crossing the seam moving right (Eq. 59)
                left = edge[i] + ((x0 == 0 && bc_x == BC_GRADIENT) ? jw : C(0));
            }
#pragma unroll
            for (int j = V - 1; j >= 1; --j) d[i][j] = d[i][j - 1];
            d[i][0] = left;
        } else {
            C right = __shfl_down_sync(0xffffffffu, d[i][0], 1);
            if (need_right) {
                // crossing the seam moving left (Eq. 60)
                right = edge[i] - ((x0 + V == nx && bc_x == BC_GRADIENT) ? jw : C(0));
            }
#pragma unroll
            for (int j = 0; j < V - 1; ++j) d[i][j] = d[i][j + 1];
            d[i][V - 1] = right;
        }
    }
    return VecPos{y, xv, x0, active, bottom, top};
}

// Loads the thread's V nodes of a stored state (no streaming): step 0.
// 16-bit storage: each value with its own tile's reference population.
template <typename T>
__device__ __forceinline__ VecPos vector_local(const T *__restrict__ src, int nx, int ny,
                                               long long plane, long long t,
                                               const Coef<typename Store<T>::C> &k,
                                               typename Store<T>::C (&d)[8][Pack<T>::V]) {
    using C = typename Store<T>::C;
    constexpr int V = Pack<T>::V;
    const int tpr = nx / V;
    const long long total = (long long)tpr * ny;
    const bool active = t < total;
    const int y = active ? int(t / tpr) : 0;
    const int xv = active ? int(t - (long long)y * tpr) : 0;
    const int x0 = xv * V;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (active) {
            Pack<T>::unpack(ld_stream(src + (long long)i * plane + (long long)y * nx + x0), d[i]);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) d[i][j] = C(0);
        }
    }
    if constexpr (sizeof(T) == 2) {
        if (active) {
            const Ref3 a = ref_of<T>(ld_ref_stored(src, k, t));     // tile t = vector t
            float R[8];
            ref_pops(a, k, R);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < V; ++j) d[i][j] = f_add(d[i][j], R[i]);
        }
    }
    return VecPos{y, xv, x0, active, false, false};
}

// 16-bit storage, node by node: collides the thread's 8 pulled nodes n[j]
// (boundaries applied), stores them (tile `tile` of dst, row offset `out`)
// less the reference populations of `enc` and writes the tile's references
// {enc, the next one from the nodes' moments} (refs16.cuh).
template <typename T, bool SR = false>
__device__ __forceinline__ void collide_store16(float (&n)[8][8], const Coef<float> &k,
                                                T *__restrict__ dst, long long plane,
                                                long long out, long long tile, uint2 enc) {
    float rho[8], mx[8], my[8], Re[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        moments_f32(n[j], rho[j], mx[j], my[j]);
        relax_f32(n[j], rho[j], mx[j], my[j], k);
    }
    ref_pops(ref_of<T>(enc), k, Re);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        unsigned wd[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)       // node pairs (2m, 2m + 1), as the pair kernels
            wd[m] = store_word<T, SR>(
                make_float2(f_sub(n[2 * m][i], Re[i]), f_sub(n[2 * m + 1][i], Re[i])),
                (unsigned)(out >> 1) + m, i);
        st_stream(dst + (long long)i * plane + out, make_uint4(wd[0], wd[1], wd[2], wd[3]));
    }
    st_ref(dst, k, tile, enc,
           next_ref<T>(tile_tree8(rho), tile_tree8(mx), tile_tree8(my), k, k.ref_gamma));
}

}  // namespace plbm
