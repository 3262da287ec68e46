// Device-side building blocks of the D2Q8 phonon lattice Boltzmann step
// (Guo & Wang, Section 2.2): storage traits, the collision on deviations,
// and the boundary rules applied to pulled populations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace plbm {

// Eq. 14 in the order Eqs. 59-60 imply; index i = the paper's direction i+1.
//   0:(1,0) 1:(0,1) 2:(-1,0) 3:(0,-1) 4:(1,1) 5:(-1,1) 6:(-1,-1) 7:(1,-1)
__host__ __device__ constexpr int cx_of(int i) {
    return (i == 0 || i == 4 || i == 7) ? 1 : (i == 2 || i == 5 || i == 6) ? -1 : 0;
}
__host__ __device__ constexpr int cy_of(int i) {
    return (i == 1 || i == 4 || i == 5) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}

enum { BC_PERIODIC = 0, BC_GRADIENT = 1, BC_WALLS = 2, BC_SIDES = 3 };
// Treatments of the sides of a BC_SIDES direction (Section 2.5).
enum { SIDE_DIFFUSE = 0, SIDE_ISOTHERMAL = 1, SIDE_HEAT_FLUX = 2 };

// Coefficients of the collision, computed on the host in FP64 and rounded
// once to the compute type C.  On deviations d_i (scaled by s), with
//   rho = sum d_i, m = sum c_i d_i, q = m - lambda m  (Eq. 54, kappa = 1 - lambda),
//   t_i = h_i (c_i . q)                      ((5/3) a_i c_i.q of Eqs. 15-16),
//   eq_i = w_i rho + t_i                     (Eq. 15 on deviations),
// the post-collision deviation is (Eq. 13 right-hand side with Eq. 16)
//   d_i* = d_i - omega (d_i - eq_i) - sigma t_i,
// omega = 1/tau, sigma = (1 - 1/(2 tau)) / tau_r.  The FP32 collision
// (relax_f32) takes the same update with the resistive term inside the
// relaxation, d_i* = d_i - omega (d_i - w_i rho - t'_i), where t'_i is t_i
// with (1 - zeta) m in place of q, zeta = lambda + sigma tau (1 - lambda), so
// that omega (1 - zeta) = omega (1 - lambda) - sigma (1 - lambda): one
// rounded coefficient for the flux factor instead of two terms.
// The rounded coefficients keep the sums the scheme conserves exact in the
// rounded values: 4 w_axis + 4 w_diag = 1, 2 h_axis + 4 h_diag = 1 and
// u_axis + 2 u_diag = 1 hold exactly (w_diag = 1/4 - w_axis and the other
// two are exact in binary floating point), and 1 - kappa is carried as
// lambda rather than recovered from a rounded kappa.  Otherwise a rounded
// coefficient would bias every step the same way and the bias would grow
// linearly with the step count.
template <typename C>
struct Coef {
    C omega, sigma, lambda;
    C zeta;                   // lambda + sigma tau (1 - lambda), the FP32 flux factor's complement
    C w_axis, w_diag;         // Eq. 17
    C h_axis, h_diag;         // (5/3) a_i, Eq. 18
    C u_axis, u_diag;         // Eq. 58: w_i / (5/18) = 4/5 and 1/10
    C jump_axis, jump_diag;   // s w_i delta_e, Eqs. 59-60
    // Sides of BC_SIDES directions, in the order left, right, bottom, top.
    int side_kind[4];         // SIDE_*
    C side_axis[4];           // isothermal: s w_i (e_s - e_ref), Eq. 55
    C side_diag[4];
    C side_flux[4];           // heat flux: s q_0 (2 tau_r + 1)/(2 tau_r), Eq. 57
    // 16-bit storage only (refs16.cuh): populations are stored relative to a
    // reference equilibrium of their tile of 2^tile_shift nodes of a row.
    int tile_shift;           // 3: tiles of 8 nodes; 0: of one node; -1: no references
    int tiles_x;              // tiles per row, nx >> tile_shift
    long long ref_off;        // element offset of the reference plane, 8 nx ny
    C rw_axis, rw_diag;       // 4 w_i, 4 h_i: reference populations from {rho, j} / 4
    C rh_axis, rh_diag;
    C ref_rho;                // 1 / (4 nodes-per-tile): tile sum of rho -> reference
    C ref_gamma;              // gamma / (4 nodes-per-tile), gamma m = post-collision flux
    int stochastic;           // 16-bit storage rounded stochastically (refs16.cuh)
};

// Storage traits: how a population plane element is stored and converted.
template <typename T> struct Store;
template <> struct Store<float> {
    using C = float;
    __device__ static C load(float v) { return v; }
    __device__ static float put(C v) { return v; }
};
template <> struct Store<double> {
    using C = double;
    __device__ static C load(double v) { return v; }
    __device__ static double put(C v) { return v; }
};
template <> struct Store<__half> {
    using C = float;
    __device__ static C load(__half v) { return __half2float(v); }
    __device__ static __half put(C v) { return __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    using C = float;
    __device__ static C load(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 put(C v) { return __float2bfloat16_rn(v); }
};

// Collision of one node, in place on the 8 pulled deviations.
template <typename C>
__device__ __forceinline__ void collide(C (&d)[8], const Coef<C> &k) {
    const C rho = ((d[0] + d[2]) + (d[1] + d[3])) + ((d[4] + d[6]) + (d[5] + d[7]));
    const C mx = (d[0] - d[2]) + (d[4] - d[6]) + (d[7] - d[5]);
    const C my = (d[1] - d[3]) + (d[4] - d[6]) + (d[5] - d[7]);
    const C qx = mx - k.lambda * mx;
    const C qy = my - k.lambda * my;
    const C wa = k.w_axis * rho;
    const C wd = k.w_diag * rho;
    // t_i for i = 0..7: c_i.q = qx, qy, -qx, -qy, qx+qy, qy-qx, -qx-qy, qx-qy
    const C ta = k.h_axis * qx;
    const C tb = k.h_axis * qy;
    const C tp = k.h_diag * (qx + qy);
    const C tm = k.h_diag * (qx - qy);
    const C t[8] = {ta, tb, -ta, -tb, tp, -tm, -tp, tm};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const C eq = (i < 4 ? wa : wd) + t[i];
        d[i] = d[i] - k.omega * (d[i] - eq) - k.sigma * t[i];
    }
}

// FP32 arithmetic with its rounding spelled out: every operation rounds once,
// in the order written, and the compiler chooses no contraction.  The same
// sequence on float (one node) and on float2 (two nodes, packed FP32 pair
// instructions, each lane rounded as the scalar operation) gives identical
// bits, so every kernel that stores the collision in FP32 or 16 bits agrees
// with every other to the bit whichever form it uses.
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 f_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b rounded once: fma(b, -1, a) (the product is exact)
__device__ __forceinline__ float2 f_sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 f_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f_fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
}
template <typename V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }

// One population's relaxation, d* = d - omega (d - eq), with eq = w rho + t_i
// formed in one rounding (fused multiply-add) and t_i = +t (plus) or -t
// (minus); t carries the flux factor 1 - zeta, which holds the resistive
// term sigma t_i of Eq. 16.  For minus the negated equilibrium
// -eq = w (-rho) + t is formed instead (rounding is symmetric, so it is
// exactly -eq) and added.
template <typename V>
__device__ __forceinline__ V relax_plus(V d, V w, V rho, V t, V neg_omega) {
    const V eq = f_fma(w, rho, t);
    return f_fma(neg_omega, f_sub(d, eq), d);
}
template <typename V>
__device__ __forceinline__ V relax_minus(V d, V w, V neg_rho, V t, V neg_omega) {
    const V neg_eq = f_fma(w, neg_rho, t);
    return f_fma(neg_omega, f_add(d, neg_eq), d);
}

// The moments of Eqs. 53-54 before the kappa factor: rho = sum d_i and
// m = sum c_i d_i, in the order every FP32 kernel forms them (15
// operations: my subtracts d_7 - d_5, which rounds to exactly minus
// d_5 - d_7, instead of adding the latter).
template <typename V>
__device__ __forceinline__ void moments_f32(const V (&d)[8], V &rho, V &mx, V &my) {
    rho = f_add(f_add(f_add(d[0], d[2]), f_add(d[1], d[3])),
                f_add(f_add(d[4], d[6]), f_add(d[5], d[7])));
    const V s46 = f_sub(d[4], d[6]);
    const V s75 = f_sub(d[7], d[5]);
    mx = f_add(f_add(f_sub(d[0], d[2]), s46), s75);
    my = f_sub(f_add(f_sub(d[1], d[3]), s46), s75);
}

// The relaxation of collide_f32 given the node's moments.
template <typename V>
__device__ __forceinline__ void relax_f32(V (&d)[8], V rho, V mx, V my, const Coef<float> &k) {
    const V neg_zeta = splat<V>(-k.zeta);
    const V qx = f_fma(neg_zeta, mx, mx);               // (1 - zeta) m
    const V qy = f_fma(neg_zeta, my, my);
    const V neg_rho = f_mul(splat<V>(-1.f), rho);       // exact
    const V wa = splat<V>(k.w_axis), wd = splat<V>(k.w_diag);
    const V ha = splat<V>(k.h_axis), hd = splat<V>(k.h_diag);
    const V ta = f_mul(ha, qx);
    const V tb = f_mul(ha, qy);
    const V tp = f_mul(hd, f_add(qx, qy));
    const V tm = f_mul(hd, f_sub(qx, qy));
    const V no = splat<V>(-k.omega);
    // t_i for i = 0..7: ta, tb, -ta, -tb, tp, -tm, -tp, tm
    d[0] = relax_plus(d[0], wa, rho, ta, no);
    d[1] = relax_plus(d[1], wa, rho, tb, no);
    d[2] = relax_minus(d[2], wa, neg_rho, ta, no);
    d[3] = relax_minus(d[3], wa, neg_rho, tb, no);
    d[4] = relax_plus(d[4], wd, rho, tp, no);
    d[5] = relax_minus(d[5], wd, neg_rho, tm, no);
    d[6] = relax_minus(d[6], wd, neg_rho, tp, no);
    d[7] = relax_plus(d[7], wd, rho, tm, no);
}

// The collision above in FP32 on one node (V = float) or on two nodes at once
// (V = float2: lane x one node, lane y the other).  Operation order chosen
// for accuracy and count (48 operations per node): over 5000 steps of the
// 4096 x 4 second-sound pulse (Kn_R = 0.1) the max error against FP64 is
// 6.2e-6 (7.1e-6 with sigma t_i as a separate term, 56 operations; 1.2e-5
// with w rho also rounded apart from t_i), and 6.6e-8 against 8.1e-7 at
// 300 steps of the 8192 x 8192 heat mode.  Folding omega into the weights
// instead (d* = (1 - omega) d + omega eq, 41 operations) loses the small
// differences d - eq: about 80 times less accurate at Kn_R = 1 and 10 on the
// second-sound pulse (FP32 emulated on the host).
template <typename V>
__device__ __forceinline__ void collide_f32(V (&d)[8], const Coef<float> &k) {
    V rho, mx, my;
    moments_f32(d, rho, mx, my);
    relax_f32(d, rho, mx, my, k);
}

// FP32 compute (FP32 and 16-bit storage): the spelled-out form.
__device__ __forceinline__ void collide(float (&d)[8], const Coef<float> &k) {
    collide_f32<float>(d, k);
}

// Eq. 58 on a wall node whose pulled incident populations are in d.
// Bottom wall (y = 0, outward normal (0,-1)): unknown 1,4,5 from incident
// 3,6,7; top wall (y = ny-1): unknown 3,6,7 from incident 1,4,5.  The sum of
// w over the unknowns is 5/18, so w_i/(5/18) is 4/5 (axis) or 1/10 (diag).
template <typename C>
__device__ __forceinline__ void wall_bottom(C (&d)[8], const Coef<C> &k) {
    const C s = d[3] + d[6] + d[7];
    d[1] = k.u_axis * s;
    d[4] = k.u_diag * s;
    d[5] = k.u_diag * s;
}
template <typename C>
__device__ __forceinline__ void wall_top(C (&d)[8], const Coef<C> &k) {
    const C s = d[1] + d[4] + d[5];
    d[3] = k.u_axis * s;
    d[6] = k.u_diag * s;
    d[7] = k.u_diag * s;
}
// The same on two nodes of one row at once (FP32 pairs; identical bits).
__device__ __forceinline__ void wall_bottom(float2 (&d)[8], const Coef<float> &k) {
    const float2 s = f_add(f_add(d[3], d[6]), d[7]);
    d[1] = f_mul(splat<float2>(k.u_axis), s);
    d[4] = f_mul(splat<float2>(k.u_diag), s);
    d[5] = d[4];
}
__device__ __forceinline__ void wall_top(float2 (&d)[8], const Coef<float> &k) {
    const float2 s = f_add(f_add(d[1], d[4]), d[5]);
    d[3] = f_mul(splat<float2>(k.u_axis), s);
    d[6] = f_mul(splat<float2>(k.u_diag), s);
    d[7] = d[6];
}

// Section 2.5 on a node of the sides of BC_SIDES directions, after the
// pull (unknown populations are 0 in d).  on_* tell which sides the node
// lies on.  A node on an isothermal side is set to the equilibrium at rest
// at e_s (Eq. 55; the first isothermal side in the order left, right,
// bottom, top when two meet at a corner).  Otherwise each of its sides, in
// the order bottom, top, left, right, sets its unknown populations
// (c_i . n < 0) to w_i / (5/18) times the sum of the incident ones
// (c_i . n > 0) plus s q_0 / kappa (Eq. 57; Eq. 58 when q_0 = 0).
template <typename C>
__device__ __forceinline__ void apply_sides(C (&d)[8], const Coef<C> &k, bool on_left,
                                            bool on_right, bool on_bottom, bool on_top) {
    bool iso = false;
    C va = C(0), vd = C(0);
    // later assignments win, so the first isothermal side in order is kept
    if (on_top && k.side_kind[3] == SIDE_ISOTHERMAL) { iso = true; va = k.side_axis[3]; vd = k.side_diag[3]; }
    if (on_bottom && k.side_kind[2] == SIDE_ISOTHERMAL) { iso = true; va = k.side_axis[2]; vd = k.side_diag[2]; }
    if (on_right && k.side_kind[1] == SIDE_ISOTHERMAL) { iso = true; va = k.side_axis[1]; vd = k.side_diag[1]; }
    if (on_left && k.side_kind[0] == SIDE_ISOTHERMAL) { iso = true; va = k.side_axis[0]; vd = k.side_diag[0]; }
    if (iso) {
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = i < 4 ? va : vd;
        return;
    }
    if (on_bottom) {          // n = (0,-1): unknown 1,4,5; incident 3,6,7
        const C s = (d[3] + d[6] + d[7]) + k.side_flux[2];
        d[1] = k.u_axis * s;
        d[4] = k.u_diag * s;
        d[5] = k.u_diag * s;
    }
    if (on_top) {             // n = (0,1): unknown 3,6,7; incident 1,4,5
        const C s = (d[1] + d[4] + d[5]) + k.side_flux[3];
        d[3] = k.u_axis * s;
        d[6] = k.u_diag * s;
        d[7] = k.u_diag * s;
    }
    if (on_left) {            // n = (-1,0): unknown 0,4,7; incident 2,5,6
        const C s = (d[2] + d[5] + d[6]) + k.side_flux[0];
        d[0] = k.u_axis * s;
        d[4] = k.u_diag * s;
        d[7] = k.u_diag * s;
    }
    if (on_right) {           // n = (1,0): unknown 2,5,6; incident 0,4,7
        const C s = (d[0] + d[4] + d[7]) + k.side_flux[1];
        d[2] = k.u_axis * s;
        d[5] = k.u_diag * s;
        d[6] = k.u_diag * s;
    }
}

// Generic pull of the 8 populations arriving at node (x, y) at the next
// step from post-collision planes (one node, any nx).  Applies the seam
// jump, the walls and the per-side treatments.  `load(i, sx, sy)` returns
// population i of node (sx, sy) in the compute type: pull_node reads global
// planes (the scalar step kernel and every read-out kernel), the cluster-
// resident kernel reads shared memory.
template <typename C, typename Load>
__device__ __forceinline__ void pull_node_with(const Load &load, int nx, int ny, int x, int y,
                                               int bc_x, int bc_y, const Coef<C> &k,
                                               C (&d)[8]) {
    const bool walls = bc_y == BC_WALLS;
    const bool sides_x = bc_x == BC_SIDES, sides_y = bc_y == BC_SIDES;
    const bool open_y = walls || sides_y;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int cx = cx_of(i), cy = cy_of(i);
        int sy = y - cy;
        if (open_y && (sy < 0 || sy >= ny)) {
            d[i] = C(0);          // unknown: filled by Eq. 58 / the sides below
            continue;
        }
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        int sx = x - cx;
        if (sides_x && (sx < 0 || sx >= nx)) {
            d[i] = C(0);          // unknown: filled by the x sides below
            continue;
        }
        C jump = C(0);
        if (sx < 0) {             // crossed the seam moving right (Eq. 59)
            sx += nx;
            if (bc_x == BC_GRADIENT) jump = (i < 4) ? k.jump_axis : k.jump_diag;
        } else if (sx >= nx) {    // crossed the seam moving left (Eq. 60)
            sx -= nx;
            if (bc_x == BC_GRADIENT) jump = -((i < 4) ? k.jump_axis : k.jump_diag);
        }
        d[i] = load(i, sx, sy) + jump;
    }
    if (walls) {
        if (y == 0) wall_bottom(d, k);
        if (y == ny - 1) wall_top(d, k);
    }
    if (sides_x || sides_y)
        apply_sides(d, k, sides_x && x == 0, sides_x && x == nx - 1, sides_y && y == 0,
                    sides_y && y == ny - 1);
}

// Residual contribution of one node of the state at step n (pulled, after
// the boundary, before collision), in the compute type C.  de = e - e_ref and
// q are added to the thread's partial sums loc (in node order) and compared
// with / replace the node's history values (de, qx, qy at the previous
// residual) held in h_de, h_qx, h_qy:
//   loc[0] += de, loc[1] += de^2, loc[2] += |q|^2,
//   loc[3] += |(de, q) - history|^2, loc[4] += 1 if a value is not finite.
// warp_flush_residual then sums loc over the warp in C (a fixed shuffle
// order) and adds the warp's sums to FP64 accumulators.  FP64 arithmetic
// runs at a small fraction of the FP32 rate on this GPU, so it is kept to
// one conversion and add per warp and quantity.
template <typename C>
__device__ __forceinline__ void residual_terms(const C (&d)[8], const Coef<C> &k, C inv_s,
                                               C &h_de, C &h_qx, C &h_qy, bool have_prev,
                                               C (&loc)[5]) {
    const C rho = ((d[0] + d[2]) + (d[1] + d[3])) + ((d[4] + d[6]) + (d[5] + d[7]));
    const C mx = (d[0] - d[2]) + (d[4] - d[6]) + (d[7] - d[5]);
    const C my = (d[1] - d[3]) + (d[4] - d[6]) + (d[5] - d[7]);
    const C de = rho * inv_s;
    const C qx = (mx - k.lambda * mx) * inv_s;
    const C qy = (my - k.lambda * my) * inv_s;
    if (!(isfinite(de) && isfinite(qx) && isfinite(qy))) loc[4] += C(1);
    loc[0] += de;
    loc[1] += de * de;
    loc[2] += qx * qx + qy * qy;
    if (have_prev) {
        const C a = de - h_de, b = qx - h_qx, c = qy - h_qy;
        loc[3] += a * a + b * b + c * c;
    }
    h_de = de;
    h_qx = qx;
    h_qy = qy;
}

// Same for one node whose history lives in the planes prev (3 x n of C).
template <typename C>
__device__ __forceinline__ void residual_node(const C (&d)[8], const Coef<C> &k, C inv_s,
                                              C *__restrict__ prev, long long n,
                                              long long node, bool have_prev, C (&loc)[5]) {
    C h0 = have_prev ? prev[node] : C(0);
    C h1 = have_prev ? prev[n + node] : C(0);
    C h2 = have_prev ? prev[2 * n + node] : C(0);
    residual_terms(d, k, inv_s, h0, h1, h2, have_prev, loc);
    prev[node] = h0;
    prev[n + node] = h1;
    prev[2 * n + node] = h2;
}

// Sums loc over the (full) warp in C, adds the totals to acc in lane 0 and
// clears loc.  Every lane of the warp must call it.
template <typename C>
__device__ __forceinline__ void warp_flush_residual(C (&loc)[5], double (&acc)[5]) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        C v = loc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) acc[q] += (double)v;
        loc[q] = C(0);
    }
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of 5 doubles per thread (every thread of the block must
// call it); thread 0 writes the block's sums to out[0..4].
__device__ __forceinline__ void block_sum5_store(const double (&v)[5], double *out) {
    __shared__ double sh[5][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double w = warp_sum_f64(v[q]);
        if (lane == 0) sh[q][warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double w = warp_sum_f64(lane < nw ? sh[q][lane] : 0.0);
            if (lane == 0) out[q] = w;
        }
    }
}

// Block-wide sum when only lane 0 of each warp holds values (after
// warp_flush_residual): no FP64 shuffles; thread 0 adds the warps' values in
// warp order and writes out[0..4].  Every thread must call it.
__device__ __forceinline__ void block_sum5_lane0(const double (&v)[5], double *out) {
    __shared__ double sh[5][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) sh[q][warp] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[q][w];
            out[q] = s;
        }
    }
}

// Request for the fused residual in a step launch.
template <typename C>
struct ResidualReq {
    C *prev;            // history planes (3 x n of C), read and overwritten
    int have_prev;      // compare with the history
    C inv_scale;        // 1 / storage scale
    double *partials;   // 5 doubles per block of the launch
};

}  // namespace plbm
