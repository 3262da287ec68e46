// Initialisation and read-out kernels: the Eq. 15 initial state, moments
// (Eqs. 53-54), raw populations, and the residual / energy reduction.  None
// is on the per-step path.  Per-node arithmetic runs in the compute type C
// (FP64 arithmetic is slow on this GPU); only the FP64 outputs and the
// per-warp sums of the reduction are formed in double.
#include "lbm_kernels.h"
#include "vector_pull.cuh"

namespace plbm {

// Populations of the state at the current step for node (x, y), as the
// stream-collide kernel sees them before colliding.
template <typename T>
__device__ __forceinline__ void state_node(const T *__restrict__ src, const Readout &r,
                                           const Coef<typename Store<T>::C> &k, int x, int y,
                                           typename Store<T>::C (&d)[8]) {
    const long long plane = (long long)r.nx * r.ny;
    if (r.pulled) {
        pull_node<T>(src, plane, r.nx, r.ny, x, y, r.bc_x, r.bc_y, k, d);
    } else {
        const long long node = (long long)y * r.nx + x;
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = Store<T>::load(src[(long long)i * plane + node]);
        if constexpr (sizeof(T) == 2) {        // stored relative to the node's tile reference
            float R[8];
            ref_pops(ref_of<T>(ld_ref_stored(src, k, tile_of(k, x, y))), k, R);
#pragma unroll
            for (int i = 0; i < 8; ++i) d[i] = f_add(d[i], R[i]);
        }
    }
}

// e - e_ref and q of one node in the compute type (Eqs. 53-54).
template <typename C>
__device__ __forceinline__ void node_moments(const C (&d)[8], const Coef<C> &k, C inv_s, C &de,
                                             C &qx, C &qy) {
    const C rho = ((d[0] + d[2]) + (d[1] + d[3])) + ((d[4] + d[6]) + (d[5] + d[7]));
    const C mx = (d[0] - d[2]) + (d[4] - d[6]) + (d[7] - d[5]);
    const C my = (d[1] - d[3]) + (d[4] - d[6]) + (d[5] - d[7]);
    de = rho * inv_s;
    qx = (mx - k.lambda * mx) * inv_s;
    qy = (my - k.lambda * my) * inv_s;
}

// ---------------------------------------------------------------------------
// Scalar read-outs (any nx).  Loops are warp-uniform so warp shuffles are
// legal inside them.
template <typename T>
__global__ void moments_scalar(const T *__restrict__ src, Readout r,
                               Coef<typename Store<T>::C> k, double *e, double *qx, double *qy) {
    using C = typename Store<T>::C;
    const long long n = (long long)r.nx * r.ny;
    const C inv_s = (C)r.inv_scale;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = int(node / r.nx), x = int(node - (long long)y * r.nx);
        C d[8];
        state_node<T>(src, r, k, x, y, d);
        C de, a, b;
        node_moments(d, k, inv_s, de, a, b);
        if (e) e[node] = r.e_ref + (double)de;
        if (qx) qx[node] = (double)a;
        if (qy) qy[node] = (double)b;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
residual_scalar(const T *__restrict__ src, Readout r, Coef<typename Store<T>::C> k,
                typename Store<T>::C *__restrict__ prev, int have_prev,
                double *__restrict__ partials) {
    using C = typename Store<T>::C;
    const long long n = (long long)r.nx * r.ny;
    const C inv_s = (C)r.inv_scale;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const long long node = base + (threadIdx.x & 31);
        C loc[5] = {C(0), C(0), C(0), C(0), C(0)};
        if (node < n) {
            const int y = int(node / r.nx), x = int(node - (long long)y * r.nx);
            C d[8];
            state_node<T>(src, r, k, x, y, d);
            residual_node(d, k, inv_s, prev, n, node, have_prev != 0, loc);
        }
        warp_flush_residual(loc, acc);
    }
    block_sum5_lane0(acc, partials + (size_t)blockIdx.x * 5);
}

// ---------------------------------------------------------------------------
// Vectorised read-outs (nx % V == 0): one thread per 16-byte vector of nodes,
// the same pull (and so the same node-to-warp grouping of the residual sums)
// as the vector stream-collide kernel.
enum { READ_MOMENTS = 0, READ_RESIDUAL = 1 };

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
readout_vector(const T *__restrict__ src, Readout r, Coef<typename Store<T>::C> k, double *e,
               double *qx, double *qy, typename Store<T>::C *__restrict__ prev, int have_prev,
               double *__restrict__ partials) {
    using C = typename Store<T>::C;
    constexpr int V = Pack<T>::V;
    const long long plane = (long long)r.nx * r.ny;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const C inv_s = (C)r.inv_scale;
    C d[8][V];
    const VecPos p = r.pulled ? vector_pull<T>(src, r.nx, r.ny, plane, r.bc_x, r.bc_y, k, t, d)
                              : vector_local<T>(src, r.nx, r.ny, plane, t, k, d);
    C loc[5] = {C(0), C(0), C(0), C(0), C(0)};
    if (p.active) {
        const long long out = (long long)p.y * r.nx + p.x0;
        C n[V][8];
#pragma unroll
        for (int j = 0; j < V; ++j) {
#pragma unroll
            for (int i = 0; i < 8; ++i) n[j][i] = d[i][j];
            if (p.bottom) wall_bottom(n[j], k);
            if (p.top) wall_top(n[j], k);
            if (MODE == READ_MOMENTS) {
                C de, a, b;
                node_moments(n[j], k, inv_s, de, a, b);
                if (e) e[out + j] = r.e_ref + (double)de;
                if (qx) qx[out + j] = (double)a;
                if (qy) qy[out + j] = (double)b;
            }
        }
        if (MODE == READ_RESIDUAL)
            residual_vec<C, V>(n, k, inv_s, prev, plane, out, have_prev != 0, loc);
    }
    if (MODE == READ_RESIDUAL) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        warp_flush_residual(loc, acc);
        block_sum5_lane0(acc, partials + (size_t)blockIdx.x * 5);
    }
}

// Weights of Eq. 17, for adding back the rest-state part of a deviation.
__device__ __forceinline__ double omega_of(int i) { return i < 4 ? 2.0 / 9.0 : 1.0 / 36.0; }

template <typename T>
__global__ void populations_kernel(const T *__restrict__ src, Readout r,
                                   Coef<typename Store<T>::C> k, double *f) {
    using C = typename Store<T>::C;
    const long long n = (long long)r.nx * r.ny;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = int(node / r.nx), x = int(node - (long long)y * r.nx);
        C d[8];
        state_node<T>(src, r, k, x, y, d);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            f[(long long)i * n + node] = (double)d[i] * r.inv_scale + omega_of(i) * r.e_ref;
    }
}

// Fixed-order sum of the per-block partials (deterministic result).  One
// block of FINALIZE_THREADS; each thread sums every FINALIZE_THREADS-th
// record, four records per iteration so that enough loads are in flight for
// one SM to stream the ~2.6 MB of partials of an 8192^2 lattice.
// Block k sums records [k chunk, min((k + 1) chunk, blocks)) into out[5 k ..].
constexpr int FINALIZE_THREADS = 1024;

__global__ void __launch_bounds__(FINALIZE_THREADS)
finalize_sums(const double *__restrict__ partials, int blocks, int chunk,
              double *__restrict__ out) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int stride = FINALIZE_THREADS;
    const int first = blockIdx.x * chunk;
    const int end = min(blocks, first + chunk);
    int b = first + threadIdx.x;
    for (; b + 3 * stride < end; b += 4 * stride) {
        double v[4][5];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 5; ++q) v[u][q] = partials[(size_t)(b + u * stride) * 5 + q];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q] += v[u][q];
    }
    for (; b < end; b += stride) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += partials[(size_t)b * 5 + q];
    }
    block_sum5_store(acc, out + (size_t)blockIdx.x * 5);
}

// Eq. 15 on deviations, in the compute type: d_i = s (w_i (e - e_ref) +
// (5/3) a_i c_i.q), written as the state of step 0 into `pre` and, collided,
// into `post`.
template <typename T>
__global__ void init_kernel(const double *__restrict__ e, const double *__restrict__ qx,
                            const double *__restrict__ qy, int nx, int ny, double e_ref,
                            double scale, Coef<typename Store<T>::C> k, T *__restrict__ pre,
                            T *__restrict__ post) {
    using C = typename Store<T>::C;
    const long long n = (long long)nx * ny;
    const C s = (C)scale;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const C de = (C)(e[node] - e_ref);
        const C a = qx ? (C)qx[node] : C(0);
        const C b = qy ? (C)qy[node] : C(0);
        const C wa = k.w_axis * de, wd = k.w_diag * de;
        const C ta = k.h_axis * a, tb = k.h_axis * b;
        const C tp = k.h_diag * (a + b), tm = k.h_diag * (a - b);
        const C dv[8] = {wa + ta, wa + tb, wa - ta, wa - tb, wd + tp, wd - tm, wd - tp, wd + tm};
        C d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const T v = Store<T>::put(dv[i] * s);
            pre[(long long)i * n + node] = v;
            d[i] = Store<T>::load(v);
        }
        collide(d, k);
#pragma unroll
        for (int i = 0; i < 8; ++i) post[(long long)i * n + node] = Store<T>::put(d[i]);
    }
}

// The same for 16-bit storage, stored relative to tile references
// (refs16.cuh): the step-0 state is stored against the reference of its
// own moments, its collision against the reference of the collided state's
// moments (there is no earlier step whose reference could be used), and
// both buffers' tiles get {that reference, that reference}.  Every lane of a
// warp runs each node (tile sums over aligned lanes); lanes past the end
// work on the last node and store nothing.
template <typename T>
__global__ void init_kernel16(const double *__restrict__ e, const double *__restrict__ qx,
                              const double *__restrict__ qy, int nx, int ny, double e_ref,
                              double scale, Coef<float> k, T *__restrict__ pre,
                              T *__restrict__ post) {
    const long long n = (long long)nx * ny;
    const float s = (float)scale;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool tiles8 = k.tile_shift == 3;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const long long at = base + (threadIdx.x & 31);
        const bool valid = at < n;
        const long long node = valid ? at : n - 1;
        const int y = int(node / nx), x = int(node - (long long)y * nx);
        const bool lead = valid && (x & ((1 << k.tile_shift) - 1)) == 0;
        const long long tile = tile_of(k, x, y);
        const float de = (float)(e[node] - e_ref);
        const float a = qx ? (float)qx[node] : 0.f;
        const float b = qy ? (float)qy[node] : 0.f;
        const float wa = k.w_axis * de, wd = k.w_diag * de;
        const float ta = k.h_axis * a, tb = k.h_axis * b;
        const float tp = k.h_diag * (a + b), tm = k.h_diag * (a - b);
        const float dv[8] = {wa + ta, wa + tb, wa - ta, wa - tb, wd + tp, wd - tm, wd - tp, wd + tm};
        float d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = dv[i] * s;
        float rho, mx, my;
        moments_f32(d, rho, mx, my);
        if (tiles8) {
            rho = tile_tree_lanes(rho);
            mx = tile_tree_lanes(mx);
            my = tile_tree_lanes(my);
        }
        // a state before collision: its reference flux is its own first moment
        const uint2 rpre = next_ref<T>(rho, mx, my, k, k.ref_rho);
        float R[8];
        ref_pops(ref_of<T>(rpre), k, R);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const T v = Store<T>::put(f_sub(d[i], R[i]));
            if (valid) pre[(long long)i * n + node] = v;
            d[i] = f_add(Store<T>::load(v), R[i]);        // the state as the read-outs see it
        }
        if (lead) st_ref(pre, k, tile, rpre, rpre);
        moments_f32(d, rho, mx, my);
        float sr = rho, sx = mx, sy = my;
        if (tiles8) {
            sr = tile_tree_lanes(sr);
            sx = tile_tree_lanes(sx);
            sy = tile_tree_lanes(sy);
        }
        relax_f32(d, rho, mx, my, k);
        const uint2 rpost = next_ref<T>(sr, sx, sy, k, k.ref_gamma);
        ref_pops(ref_of<T>(rpost), k, R);
        if (valid) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                post[(long long)i * n + node] = Store<T>::put(f_sub(d[i], R[i]));
        }
        if (lead) st_ref(post, k, tile, rpost, rpost);
    }
}

// Largest per-node bound (2/9)|e - e_ref| + (1/3)(|qx| + |qy|) >= max |d_i|
// (unscaled), in FP32, maxed per warp; non-finite input -> +inf.
__global__ void max_deviation_kernel(const double *__restrict__ e, const double *__restrict__ qx,
                                     const double *__restrict__ qy, long long n, double e_ref,
                                     unsigned long long *out) {
    float m = 0.f;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        float v = (2.0f / 9.0f) * fabsf((float)(e[node] - e_ref));
        if (qx) v += fabsf((float)qx[node]) / 3.0f;
        if (qy) v += fabsf((float)qy[node]) / 3.0f;
        m = isfinite(v) ? fmaxf(m, v) : INFINITY;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, (unsigned long long)__double_as_longlong((double)m));
}

static unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    return (unsigned)(b > 0 ? b : 1);
}

// the vectorised pull knows the periodic, seam and wall rules but not the
// per-side treatments of BC_SIDES directions
static bool vector_readout(int precision_width, int nx, int bc_x, int bc_y) {
    return nx % precision_width == 0 && bc_x != BC_SIDES && bc_y != BC_SIDES;
}

template <typename T> static bool vec_ok(const Readout &r) {
    return vector_readout(Pack<T>::V, r.nx, r.bc_x, r.bc_y);
}

template <typename T> static unsigned vec_blocks(const Readout &r) {
    const long long threads = (long long)r.nx * r.ny / Pack<T>::V;
    return (unsigned)((threads + 255) / 256);
}

long long readout_blocks(int precision, int nx, int ny, int bc_x, int bc_y) {
    const long long plane = (long long)nx * ny;
    const int v = vector_width(precision);
    if (!vector_readout(v, nx, bc_x, bc_y)) return RESIDUAL_BLOCKS;
    return (plane / v + 255) / 256;
}

template <typename T>
cudaError_t launch_moments(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                           double *e, double *qx, double *qy, cudaStream_t stream) {
    if (vec_ok<T>(r))
        readout_vector<T, READ_MOMENTS><<<vec_blocks<T>(r), 256, 0, stream>>>(
            src, r, k, e, qx, qy, nullptr, 0, nullptr);
    else
        moments_scalar<T><<<grid_for((long long)r.nx * r.ny, 256), 256, 0, stream>>>(src, r, k,
                                                                                   e, qx, qy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_populations(const T *src, const Readout &r,
                               const Coef<typename Store<T>::C> &k, double *f,
                               cudaStream_t stream) {
    populations_kernel<T><<<grid_for((long long)r.nx * r.ny, 256), 256, 0, stream>>>(src, r, k,
                                                                                   f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const T *src, const Readout &r, const Coef<typename Store<T>::C> &k,
                            typename Store<T>::C *prev, bool have_prev, double *partials,
                            double *sums, cudaStream_t stream, double *mid) {
    int blocks;
    if (vec_ok<T>(r)) {
        blocks = (int)vec_blocks<T>(r);
        readout_vector<T, READ_RESIDUAL><<<blocks, 256, 0, stream>>>(
            src, r, k, nullptr, nullptr, nullptr, prev, have_prev ? 1 : 0, partials);
    } else {
        blocks = RESIDUAL_BLOCKS;
        residual_scalar<T><<<blocks, 256, 0, stream>>>(src, r, k, prev, have_prev ? 1 : 0,
                                                       partials);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_finalize(partials, blocks, sums, stream, mid);
}

cudaError_t launch_finalize(const double *partials, int blocks, double *sums,
                            cudaStream_t stream, double *mid, int *launches) {
    if (mid && blocks > FINALIZE_SPLIT) {
        const int chunk = (blocks + FINALIZE_MID - 1) / FINALIZE_MID;
        const int parts = (blocks + chunk - 1) / chunk;
        finalize_sums<<<parts, FINALIZE_THREADS, 0, stream>>>(partials, blocks, chunk, mid);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        finalize_sums<<<1, FINALIZE_THREADS, 0, stream>>>(mid, parts, parts, sums);
        if (launches) *launches = 2;
    } else {
        finalize_sums<<<1, FINALIZE_THREADS, 0, stream>>>(partials, blocks, blocks, sums);
        if (launches) *launches = 1;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init(const double *e, const double *qx, const double *qy, int nx, int ny,
                        double e_ref, double scale, const Coef<typename Store<T>::C> &k, T *pre,
                        T *post, cudaStream_t stream) {
    if constexpr (sizeof(T) == 2)
        init_kernel16<T><<<grid_for((long long)nx * ny, 256), 256, 0, stream>>>(
            e, qx, qy, nx, ny, e_ref, scale, k, pre, post);
    else
        init_kernel<T><<<grid_for((long long)nx * ny, 256), 256, 0, stream>>>(
            e, qx, qy, nx, ny, e_ref, scale, k, pre, post);
    return cudaGetLastError();
}

cudaError_t launch_max_deviation(const double *e, const double *qx, const double *qy,
                                 long long n, double e_ref, unsigned long long *out,
                                 cudaStream_t stream) {
    max_deviation_kernel<<<grid_for(n, 256), 256, 0, stream>>>(e, qx, qy, n, e_ref, out);
    return cudaGetLastError();
}

#define PLBM_INSTANTIATE(T)                                                                   \
    template cudaError_t launch_moments<T>(const T *, const Readout &,                        \
                                           const Coef<Store<T>::C> &, double *, double *,     \
                                           double *, cudaStream_t);                           \
    template cudaError_t launch_populations<T>(const T *, const Readout &,                    \
                                               const Coef<Store<T>::C> &, double *,           \
                                               cudaStream_t);                                 \
    template cudaError_t launch_residual<T>(const T *, const Readout &,                       \
                                            const Coef<Store<T>::C> &, Store<T>::C *, bool,   \
                                            double *, double *, cudaStream_t, double *);      \
    template cudaError_t launch_init<T>(const double *, const double *, const double *, int,  \
                                        int, double, double, const Coef<Store<T>::C> &, T *,  \
                                        T *, cudaStream_t);

PLBM_INSTANTIATE(float)
PLBM_INSTANTIATE(double)
PLBM_INSTANTIATE(__half)
PLBM_INSTANTIATE(__nv_bfloat16)

}  // namespace plbm
