// Batched solver: many independent lattices ("instances") of uneven size and
// relaxation times advanced together, one launch per time step for all of
// them, run to steady state with per-instance residuals and retirement.
//
// Layout: the instances' population planes are packed one after another in
// two shared buffers (instance i: 8 planes of nx_i * ny_i elements starting
// at element off_i, then, with 16-bit storage, its plane of tile references,
// refs16.cuh); residual histories likewise (3 planes of the compute type per
// instance).  Work is cut into items of `tpi` threads x V nodes of
// one instance; a persistent grid walks the list of items of the instances
// still running.  Each item runs the same vectorised pull, boundary and
// collision as the single-lattice vector kernel (Eqs. 13, 15, 16, 53-54, 58,
// 59-60) with its instance's coefficients.
//
// Steady-state solve: windows of K (even) steps are captured once as a CUDA
// graph -- K-1 plain step launches, one step launch that also reduces each
// item's residual sums, a per-instance fixed-order sum, and the copy of the
// sums to pinned host memory.  Between windows the host retires instances
// whose residual stayed below the tolerance on two consecutive checks and
// uploads the shorter item list; the graph reads the list and its length
// from device memory, so it is replayed unchanged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/phonon_lbm.h"
#include "lbm_kernels.h"
#include "vector_pull.cuh"
#include "wave.cuh"

namespace plbm {
namespace {

enum { B_STEP = 0, B_STEP_RES = 1, B_RES_ONLY = 2 };

template <typename C>
struct InstDev {
    long long off;       // element offset of plane 0 in the population buffers
    long long hoff;      // element offset of the history planes
    long long plane;     // nx * ny
    int nx, ny, bc_x, bc_y;
    Coef<C> k;
};

struct Item {
    int inst;            // instance index
    int first;           // first thread (vector) index within the instance
};

struct Range {
    int inst, begin, end;   // items [begin, end) of an active instance
};

// A strip-segment of one instance for the multi-step kernel (wave.cuh).
struct WItem {
    int inst, tx, sg;
};

// Block-wide sum of per-warp values (lane 0 of each warp); reusable inside a
// block-uniform loop.
__device__ __forceinline__ void item_sum5(const double (&v)[5], double *out) {
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
    __syncthreads();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512)
batch_kernel(const T *__restrict__ src, T *__restrict__ dst,
             const InstDev<typename Store<T>::C> *__restrict__ inst,
             const Item *__restrict__ items, const int *__restrict__ n_items,
             typename Store<T>::C inv_s, typename Store<T>::C *__restrict__ hist, int have_prev,
             double *__restrict__ partials) {
    using C = typename Store<T>::C;
    constexpr int V = Pack<T>::V;
    const int count = *n_items;
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const Item item = items[it];
        const InstDev<C> I = inst[item.inst];
        const long long t = (long long)item.first + threadIdx.x;
        C d[8][V];
        uint2 enc = make_uint2(0u, 0u);   // 16-bit storage: the tile's next reference
        const VecPos p = vector_pull<T>(src + I.off, I.nx, I.ny, I.plane, I.bc_x, I.bc_y, I.k, t,
                                        d, &enc);
        C loc[5] = {C(0), C(0), C(0), C(0), C(0)};
        if (p.active) {
            const long long out = (long long)p.y * I.nx + p.x0;
            C n[V][8];
#pragma unroll
            for (int j = 0; j < V; ++j) {
#pragma unroll
                for (int i = 0; i < 8; ++i) n[j][i] = d[i][j];
                if (p.bottom) wall_bottom(n[j], I.k);
                if (p.top) wall_top(n[j], I.k);
            }
            if (MODE != B_STEP)
                residual_vec<C, V>(n, I.k, inv_s, hist + I.hoff, I.plane, out, have_prev != 0,
                                   loc);
            if (MODE != B_RES_ONLY) {
                T *o = dst + I.off;
                if constexpr (sizeof(T) == 2) {
                    collide_store16<T>(n, I.k, o, I.plane, out, t, enc);   // tile t = vector t
                } else {
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        collide(n[j], I.k);
#pragma unroll
                        for (int i = 0; i < 8; ++i) d[i][j] = n[j][i];
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        st_stream(o + (long long)i * I.plane + out, Pack<T>::pack(d[i]));
                }
            }
        }
        if (MODE != B_STEP) {
            double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            warp_flush_residual(loc, acc);
            item_sum5(acc, partials + (size_t)it * 5);
        }
    }
}

// Several steps per launch (FP32 storage): each warp marches strip-segments
// of the running instances (wave.cuh), with the instance's coefficients, a
// common halo H and rows per segment.  Persistent grid: the item count is
// read from device memory, so captured launches follow retirements.
constexpr int BW_WARPS = 1;        // one strip-segment per block, as the single-lattice kernel
constexpr int BW_SMEM = BW_WARPS * wave::RING_ELEMS * (int)sizeof(float2);

template <int K>
__global__ void __launch_bounds__(BW_WARPS * 32)
batch_wave(const float *__restrict__ src, float *__restrict__ dst,
           const InstDev<float> *__restrict__ inst, const WItem *__restrict__ items,
           const int *__restrict__ n_items, int halo, int seg_rows) {
    extern __shared__ float2 bw_ring[];
    const int count = *n_items;
    const int warps = gridDim.x * BW_WARPS;
    float2 *ring = bw_ring + (threadIdx.x >> 5) * wave::RING_ELEMS;
    for (int it = blockIdx.x * BW_WARPS + (threadIdx.x >> 5); it < count; it += warps) {
        const WItem w = items[it];
        const InstDev<float> &I = inst[w.inst];
        wave::Strip a;
        a.src = src + I.off;
        a.dst = dst + I.off;
        a.plane = I.plane;
        a.nx = I.nx;
        a.ny = I.ny;
        a.bc_x = I.bc_x;
        a.bc_y = I.bc_y;
        a.seg_rows = seg_rows;
        wave::run_strip<K, true>(a, I.k, w.tx, w.sg, halo, ring);
    }
}

// One block per active instance: fixed-order sum of its items' partials.
__global__ void __launch_bounds__(128)
batch_finalize(const double *__restrict__ partials, const Range *__restrict__ ranges,
               const int *__restrict__ n_ranges, double *__restrict__ sums) {
    if ((int)blockIdx.x >= *n_ranges) return;
    const Range r = ranges[blockIdx.x];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = r.begin + threadIdx.x; b < r.end; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += partials[(size_t)b * 5 + q];
    }
    block_sum5_store(acc, sums + (size_t)r.inst * 5);
}

// Normalised steady profiles of one channel instance from its moment fields
// (device doubles [ny][nx]): for output point j of P = 256 at Y = j/(P-1),
// linear interpolation between rows y0 and y0 + 1 of the row means of
//   Q = q_x nx / ((5/9) tau_R delta_e)     (heat flux over the Fourier flux)
//   E = (e + delta_e (x - (nx-1)/2) / nx - e_ref) nx / delta_e   (e minus
//        its x-affine part, in units of the drop per cell delta_e / nx).
// Both are set by the temperature gradient alone, so a channel's profile
// does not depend on its length.
// One block per output point; out[0..P) = Q, out[P..2P) = E.
constexpr int PROFILE_POINTS = 256;

__global__ void __launch_bounds__(128)
channel_profile(const double *__restrict__ e, const double *__restrict__ qx, int nx, int ny,
                double e_ref, double delta_e, double q_unit, float *__restrict__ out) {
    const int j = blockIdx.x;
    const double yf = (double)j / (PROFILE_POINTS - 1) * (ny - 1);
    int y0 = (int)floor(yf);
    if (y0 > ny - 1) y0 = ny - 1;
    const int y1 = y0 + 1 < ny ? y0 + 1 : y0;
    const double w = yf - y0;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const double aff = delta_e * ((double)x - 0.5 * (nx - 1)) / nx;
        acc[0] += qx[(long long)y0 * nx + x];
        acc[1] += qx[(long long)y1 * nx + x];
        acc[2] += e[(long long)y0 * nx + x] + aff - e_ref;
        acc[3] += e[(long long)y1 * nx + x] + aff - e_ref;
    }
    __shared__ double res[5];
    block_sum5_store(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double q = ((1.0 - w) * res[0] + w * res[1]) / nx;
        const double ed = ((1.0 - w) * res[2] + w * res[3]) / nx;
        out[j] = (float)(q / q_unit);
        out[PROFILE_POINTS + j] = (float)(ed * nx / delta_e);
    }
}

// Interpolated value of a 256-point profile at row y of ny.
__device__ __forceinline__ double profile_at(const float *__restrict__ p, int y, int ny) {
    const double t = ny > 1 ? (double)y / (ny - 1) * (PROFILE_POINTS - 1) : 0.0;
    int j0 = (int)floor(t);
    if (j0 > PROFILE_POINTS - 2) j0 = PROFILE_POINTS - 2;
    const double w = t - j0;
    return (1.0 - w) * p[j0] + w * p[j0 + 1];
}

// Mean over the ny rows of the interpolated E profile (one block).  The
// channel conserves its total energy, so the steady state keeps the starting
// mean; removing this mean makes a profile start reach the same steady
// state as the cold start e = e_ref.
__global__ void __launch_bounds__(128)
profile_e_mean(const float *__restrict__ prof, int ny, double *__restrict__ out) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int y = threadIdx.x; y < ny; y += blockDim.x)
        acc[0] += profile_at(prof + PROFILE_POINTS, y, ny);
    __shared__ double res[5];
    block_sum5_store(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) *out = res[0] / ny;
}

// Initial fields of one channel from its predicted profile (same
// normalisation as channel_profile): q_x = Q(Y) q_unit, q_y = 0,
// e = e_ref + (delta_e / nx) (E(Y) - mean E - (x - (nx-1)/2)), Y = y/(ny-1).
__global__ void channel_fields(const float *__restrict__ prof, int nx, int ny, double e_ref,
                               double delta_e, double q_unit, const double *__restrict__ e_mean,
                               double *__restrict__ e, double *__restrict__ qx,
                               double *__restrict__ qy) {
    const long long n = (long long)nx * ny;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(node / nx), x = (int)(node - (long long)y * nx);
        const double Q = profile_at(prof, y, ny);
        const double E = profile_at(prof + PROFILE_POINTS, y, ny) - *e_mean;
        e[node] = e_ref + delta_e / nx * (E - ((double)x - 0.5 * (nx - 1)));
        qx[node] = Q * q_unit;
        qy[node] = 0.0;
    }
}

// out[i] += a v[i]
__global__ void add_scaled(float *__restrict__ out, const float *__restrict__ v, float a,
                           long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = out[i] + a * v[i];
}

}  // namespace
}  // namespace plbm

using namespace plbm;

struct lbm_batch {
    int device = 0;
    int count = 0;
    int precision = 0;
    double e_ref = 1.0;
    double scale = 1.0;
    cudaStream_t stream = nullptr;
    std::vector<lbm_instance> inst;
    std::vector<long long> off, hoff;
    long long total = 0, htotal = 0, max_plane = 0;
    void *buf[2] = {nullptr, nullptr};
    void *hist = nullptr;
    void *dinst = nullptr;           // InstDev<C>[count]
    Item *ditems = nullptr;
    Range *dranges = nullptr;
    int *dcounts = nullptr;          // [0] items, [1] ranges
    double *partials = nullptr;      // 5 per item
    double *dsums = nullptr;         // 5 per instance
    double *hsums = nullptr;         // pinned host copy
    Item *hitems = nullptr;          // pinned host staging
    Range *hranges = nullptr;
    int *hcounts = nullptr;
    long long max_items = 0;
    int n_items = 0, n_ranges = 0;
    double *fields = nullptr;        // init staging, 3 x max_plane doubles
    unsigned long long *maxbits = nullptr;
    int cur = 0;
    bool initialised = false;
    std::vector<char> active;
    std::vector<int> icur;           // buffer parity of each instance's last step
    std::vector<long> steps;
    std::vector<long> prev_step;
    std::vector<int> good;
    std::vector<double> last_r;
    bool have_prev = false;
    int tpi = 256;                   // threads per work item
    int ctas_per_sm = 0;             // 0 = as many as fit
    int grid = 0;
    int sms = 0;
    // multi-step launches (FP32): steps per launch (0: one step per launch),
    // rows per segment, strip-segment items of the running instances
    int wave_steps = 0;
    int wave_rows = 128;
    WItem *dwitems = nullptr, *hwitems = nullptr;
    long long max_witems = 0;
    int n_witems = 0;
    int wave_grid[WAVE_MAX_STEPS + 1] = {0};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // per starting buffer
    int graph_k = 0;
    std::string err;
};

namespace {

size_t elem_size(int p) { return p == PREC_FP32 ? 4 : p == PREC_FP64 ? 8 : 2; }
size_t csize(int p) { return p == PREC_FP64 ? 8 : 4; }

lbm_status bfail(lbm_batch *b, lbm_status s, const std::string &m) {
    if (b) b->err = m;
    else set_global_error(m.c_str());
    return s;
}

lbm_status bcuda(lbm_batch *b, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    (void)cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, m);
}

#define BCK(b, call)                                              \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);        \
    } while (0)

struct BGuard {
    int old = -1;
    explicit BGuard(int dev) {
        if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
        else old = -1;
    }
    ~BGuard() {
        if (old >= 0) cudaSetDevice(old);
    }
};

struct Params {
    double tau, tau_r, sigma, lambda, kappa;
};

Params params_of(const lbm_instance &in) {
    Params p;
    const double inv_c = (std::isinf(in.tau_N) ? 0.0 : 1.0 / in.tau_N) +
                         (std::isinf(in.tau_R) ? 0.0 : 1.0 / in.tau_R);
    p.tau = 1.0 / inv_c + 0.5;                                        // Eq. 49
    p.tau_r = in.tau_R;
    p.sigma = std::isinf(in.tau_R) ? 0.0 : (1.0 - 1.0 / (2.0 * p.tau)) / in.tau_R;   // Eq. 16
    p.lambda = std::isinf(in.tau_R) ? 0.0 : 1.0 / (2.0 * in.tau_R + 1.0);         // Eq. 54
    p.kappa = 1.0 - p.lambda;
    return p;
}

template <typename C>
Coef<C> coef_of(const lbm_instance &in, double scale, int precision) {
    const Params p = params_of(in);
    Coef<C> k{};
    k.omega = (C)(1.0 / p.tau);
    k.sigma = (C)p.sigma;
    k.lambda = (C)p.lambda;
    k.zeta = (C)(p.lambda + p.sigma * p.tau * (1.0 - p.lambda));
    k.w_axis = (C)(2.0 / 9.0);
    k.w_diag = (C)0.25 - k.w_axis;
    k.h_axis = (C)(1.0 / 3.0);
    k.h_diag = ((C)1 - (C)2 * k.h_axis) / (C)4;
    k.u_axis = (C)0.8;
    k.u_diag = ((C)1 - k.u_axis) / (C)2;
    k.jump_axis = (C)(scale * (2.0 / 9.0) * in.bc.delta_e);
    k.jump_diag = (C)(scale * (1.0 / 36.0) * in.bc.delta_e);
    set_tile_refs(k, precision, in.nx, in.ny, p.tau, p.tau_r);
    return k;
}

int vec_width(int p) { return vector_width(p); }

// Upload the instance table (coefficients depend on the storage scale).
template <typename C>
cudaError_t upload_table(lbm_batch *b) {
    std::vector<InstDev<C>> t(b->count);
    for (int i = 0; i < b->count; ++i) {
        const lbm_instance &in = b->inst[i];
        t[i].off = b->off[i];
        t[i].hoff = b->hoff[i];
        t[i].plane = (long long)in.nx * in.ny;
        t[i].nx = in.nx;
        t[i].ny = in.ny;
        t[i].bc_x = in.bc.x;
        t[i].bc_y = in.bc.y;
        t[i].k = coef_of<C>(in, b->scale, b->precision);
    }
    cudaError_t e = cudaMemcpyAsync(b->dinst, t.data(), sizeof(InstDev<C>) * b->count,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
}

cudaError_t upload_table_any(lbm_batch *b) {
    return b->precision == PREC_FP64 ? upload_table<double>(b) : upload_table<float>(b);
}

// Strip-segments of an instance for the multi-step launches of this batch:
// halo of the largest launch, strips of 64 - 2 halo columns.
int wave_halo(const lbm_batch *b) { return wave::halo(b->wave_steps); }
long long wave_tiles(const lbm_batch *b, const lbm_instance &in) {
    const int S = wave::stride_of(wave_halo(b));
    return (in.nx + S - 1) / S;
}
long long wave_segs(const lbm_batch *b, const lbm_instance &in) {
    const int rows = b->wave_rows < in.ny ? b->wave_rows : in.ny;
    return (in.ny + rows - 1) / rows;
}

// Items and ranges of the active instances, uploaded for the next launches.
cudaError_t rebuild_items(lbm_batch *b) {
    const int V = vec_width(b->precision);
    int ni = 0, nr = 0, nw = 0;
    for (int i = 0; i < b->count; ++i) {
        if (!b->active[i]) continue;
        const long long threads = (long long)b->inst[i].nx * b->inst[i].ny / V;
        const int begin = ni;
        for (long long f = 0; f < threads; f += b->tpi) b->hitems[ni++] = Item{i, (int)f};
        b->hranges[nr++] = Range{i, begin, ni};
        if (b->wave_steps > 0) {
            // strips of one segment next to each other (their halo columns
            // are read from L2 by both)
            const long long tiles = wave_tiles(b, b->inst[i]), segs = wave_segs(b, b->inst[i]);
            for (long long sg = 0; sg < segs; ++sg)
                for (long long tx = 0; tx < tiles; ++tx)
                    b->hwitems[nw++] = WItem{i, (int)tx, (int)sg};
        }
    }
    b->n_items = ni;
    b->n_ranges = nr;
    b->n_witems = nw;
    b->hcounts[0] = ni;
    b->hcounts[1] = nr;
    b->hcounts[2] = nw;
    cudaError_t e = cudaSuccess;
    if (ni) e = cudaMemcpyAsync(b->ditems, b->hitems, sizeof(Item) * ni, cudaMemcpyHostToDevice,
                                b->stream);
    if (e == cudaSuccess && nr)
        e = cudaMemcpyAsync(b->dranges, b->hranges, sizeof(Range) * nr, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && nw)
        e = cudaMemcpyAsync(b->dwitems, b->hwitems, sizeof(WItem) * nw, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->dcounts, b->hcounts, 3 * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    // the host staging arrays are reused by the next rebuild: wait here
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
}

template <typename T>
cudaError_t launch_mode(lbm_batch *b, int mode, int src, cudaStream_t s) {
    using C = typename Store<T>::C;
    const T *in = (const T *)b->buf[src];
    T *out = (T *)b->buf[1 - src];
    const auto *tab = (const InstDev<C> *)b->dinst;
    const C inv_s = (C)(1.0 / b->scale);
    const int hp = b->have_prev ? 1 : 0;
    if (mode == B_STEP)
        batch_kernel<T, B_STEP><<<b->grid, b->tpi, 0, s>>>(in, out, tab, b->ditems, b->dcounts,
                                                          inv_s, (C *)b->hist, hp, b->partials);
    else if (mode == B_STEP_RES)
        batch_kernel<T, B_STEP_RES><<<b->grid, b->tpi, 0, s>>>(
            in, out, tab, b->ditems, b->dcounts, inv_s, (C *)b->hist, hp, b->partials);
    else
        batch_kernel<T, B_RES_ONLY><<<b->grid, b->tpi, 0, s>>>(
            in, out, tab, b->ditems, b->dcounts, inv_s, (C *)b->hist, hp, b->partials);
    return cudaGetLastError();
}

cudaError_t launch_any(lbm_batch *b, int mode, int src, cudaStream_t s) {
    switch (b->precision) {
        case PREC_FP32: return launch_mode<float>(b, mode, src, s);
        case PREC_FP64: return launch_mode<double>(b, mode, src, s);
        case PREC_FP16: return launch_mode<__half>(b, mode, src, s);
        default: return launch_mode<__nv_bfloat16>(b, mode, src, s);
    }
}

template <int K>
cudaError_t launch_wave_k(lbm_batch *b, int src, cudaStream_t s) {
    if (!b->wave_grid[K]) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_wave<K>,
                                                                      BW_WARPS * 32, BW_SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        b->wave_grid[K] = b->sms * per_sm;
    }
    batch_wave<K><<<b->wave_grid[K], BW_WARPS * 32, BW_SMEM, s>>>(
        (const float *)b->buf[src], (float *)b->buf[1 - src], (const InstDev<float> *)b->dinst,
        b->dwitems, b->dcounts + 2, wave_halo(b), b->wave_rows);
    return cudaGetLastError();
}

// One multi-step launch of k steps (2 <= k <= wave_steps) from buffer src.
cudaError_t launch_wave(lbm_batch *b, int k, int src, cudaStream_t s) {
    switch (k) {
        case 2: return launch_wave_k<2>(b, src, s);
        case 3: return launch_wave_k<3>(b, src, s);
        case 4: return launch_wave_k<4>(b, src, s);
        case 5: return launch_wave_k<5>(b, src, s);
        case 6: return launch_wave_k<6>(b, src, s);
        case 7: return launch_wave_k<7>(b, src, s);
        default: return launch_wave_k<8>(b, src, s);
    }
}

// Steps of the next launch when m plain steps are left: up to wave_steps
// in one multi-step launch, one for a remainder of one (or without them).
int next_launch_steps(const lbm_batch *b, long m) {
    if (b->wave_steps >= WAVE_MIN_STEPS && m >= WAVE_MIN_STEPS)
        return (int)(m < b->wave_steps ? m : b->wave_steps);
    return 1;
}

// Launches n plain steps take (the buffers swap once per launch).
long plain_launches(const lbm_batch *b, long n) {
    long count = 0;
    for (long m = n; m > 0; m -= next_launch_steps(b, m)) ++count;
    return count;
}

// n plain steps from buffer *src (which follows the launches).
cudaError_t plain_steps(lbm_batch *b, long n, int *src, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (long m = n; m > 0 && e == cudaSuccess;) {
        const int k = next_launch_steps(b, m);
        e = k == 1 ? launch_any(b, B_STEP, *src, s) : launch_wave(b, k, *src, s);
        *src = 1 - *src;
        m -= k;
    }
    return e;
}

cudaError_t launch_finalize_batch(lbm_batch *b, cudaStream_t s) {
    batch_finalize<<<b->count, 128, 0, s>>>(b->partials, b->dranges, b->dcounts + 1, b->dsums);
    return cudaGetLastError();
}

template <typename T>
cudaError_t occupancy(int tpi, int *per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<T, B_STEP>, tpi, 0);
}

cudaError_t plan_grid(lbm_batch *b) {
    int per_sm = 0;
    cudaError_t e;
    switch (b->precision) {
        case PREC_FP32: e = occupancy<float>(b->tpi, &per_sm); break;
        case PREC_FP64: e = occupancy<double>(b->tpi, &per_sm); break;
        case PREC_FP16: e = occupancy<__half>(b->tpi, &per_sm); break;
        default: e = occupancy<__nv_bfloat16>(b->tpi, &per_sm); break;
    }
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (b->ctas_per_sm > 0 && b->ctas_per_sm < per_sm) per_sm = b->ctas_per_sm;
    b->grid = b->sms * per_sm;
    return cudaSuccess;
}

void drop_graph(lbm_batch *b) {
    for (int i = 0; i < 2; ++i) {
        if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
        b->graph[i] = nullptr;
    }
    b->graph_k = 0;
}

// Residual of every instance from the 5 sums (same formulas as lbm_residual).
void finish(lbm_batch *b, int i, const double *s, double *r_out) {
    const lbm_instance &in = b->inst[i];
    const double n = (double)in.nx * in.ny;
    const double mean = s[0] / n;
    const double var_e = std::fmax(s[1] - n * mean * mean, 0.0);
    const double denom = std::sqrt(var_e + s[2]);
    const long k = b->steps[i] - b->prev_step[i];
    double r = INFINITY;
    if (b->have_prev && k > 0) {
        const double num = std::sqrt(s[3]);
        r = denom > 0.0 ? num / ((double)k * denom) : (num == 0.0 ? 0.0 : INFINITY);
    }
    if (s[4] > 0.0) r = NAN;
    b->prev_step[i] = b->steps[i];
    b->last_r[i] = r;
    if (r_out) *r_out = r;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_instance *inst, int count, lbm_precision precision,
                            double e_ref, void *stream, lbm_batch **out) {
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!inst || count < 1) return bfail(nullptr, LBM_EINVAL, "need at least one instance");
    if (precision < LBM_FP32 || precision > LBM_FP64)
        return bfail(nullptr, LBM_EINVAL, "unknown precision");
    if (!std::isfinite(e_ref)) return bfail(nullptr, LBM_EINVAL, "e_ref is not finite");
    const int V = vec_width(precision);
    for (int i = 0; i < count; ++i) {
        const lbm_instance &in = inst[i];
        const std::string at = "instance " + std::to_string(i) + ": ";
        if (in.nx < V || in.nx % V || in.ny < 1)
            return bfail(nullptr, LBM_EINVAL,
                         at + "nx must be a positive multiple of " + std::to_string(V));
        if ((in.bc.x != LBM_BC_PERIODIC && in.bc.x != LBM_BC_PERIODIC_GRADIENT) ||
            (in.bc.y != LBM_BC_PERIODIC && in.bc.y != LBM_BC_DIFFUSE_WALLS))
            return bfail(nullptr, in.bc.x == LBM_BC_DIFFUSE_WALLS ||
                                          in.bc.y == LBM_BC_PERIODIC_GRADIENT ||
                                          in.bc.x == LBM_BC_SIDES || in.bc.y == LBM_BC_SIDES
                                      ? LBM_EUNSUPPORTED
                                      : LBM_EINVAL,
                         at + "unsupported boundary kinds");
        if (in.bc.y == LBM_BC_DIFFUSE_WALLS && in.ny < 2)
            return bfail(nullptr, LBM_EINVAL, at + "walls need ny >= 2");
        if (!std::isfinite(in.bc.delta_e)) return bfail(nullptr, LBM_EINVAL, at + "delta_e");
        if (std::isnan(in.tau_N) || std::isnan(in.tau_R) || !(in.tau_N > 0) || !(in.tau_R > 0) ||
            (std::isinf(in.tau_N) && std::isinf(in.tau_R)))
            return bfail(nullptr, LBM_EINVAL, at + "tau_N and tau_R must be > 0, not both inf");
    }
    lbm_batch *b = new lbm_batch();
    auto bail = [&](lbm_status s) {
        lbm_batch_destroy(b);
        return s;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return bfail(nullptr, LBM_ECUDA, "cudaGetDevice failed");
    }
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->count = count;
    b->precision = precision;
    b->e_ref = e_ref;
    b->stream = (cudaStream_t)stream;
    b->inst.assign(inst, inst + count);
    b->off.resize(count);
    b->hoff.resize(count);
    for (int i = 0; i < count; ++i) {
        const long long n = (long long)inst[i].nx * inst[i].ny;
        b->off[i] = b->total;
        b->hoff[i] = b->htotal;
        b->total += state_elems(precision, inst[i].nx, inst[i].ny);
        b->htotal += 3 * n;
        b->max_plane = std::max(b->max_plane, n);
        b->max_items += (n / V + 127) / 128;     // items of at least 128 threads
    }
    b->active.assign(count, 1);
    b->icur.assign(count, 0);
    b->steps.assign(count, 0);
    b->prev_step.assign(count, 0);
    b->good.assign(count, 0);
    b->last_r.assign(count, INFINITY);
    const size_t es = elem_size(precision);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&b->buf[i], es * b->total);
    if (e == cudaSuccess) e = cudaMalloc(&b->hist, csize(precision) * b->htotal);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->dinst, (int)precision == PREC_FP64 ? sizeof(InstDev<double>) * count
                                                         : sizeof(InstDev<float>) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->ditems, sizeof(Item) * b->max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->dranges, sizeof(Range) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->dcounts, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->partials, sizeof(double) * 5 * b->max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->dsums, sizeof(double) * 5 * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->fields, sizeof(double) * 3 * b->max_plane);
    if (e == cudaSuccess) e = cudaMalloc(&b->maxbits, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&b->hsums, sizeof(double) * 5 * count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->hitems, sizeof(Item) * b->max_items);
    if (e == cudaSuccess) e = cudaMallocHost(&b->hranges, sizeof(Range) * count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->hcounts, 4 * sizeof(int));
    if (e == cudaSuccess) {
        // strip-segments of the smallest strips and segments a batch may use
        long long nw = 0;
        for (int i = 0; i < count; ++i) {
            const int S = wave::stride_of(wave::halo(WAVE_MAX_STEPS));
            nw += (long long)((inst[i].nx + S - 1) / S) * inst[i].ny;
        }
        b->max_witems = nw;
        if (precision == PREC_FP32) {
            e = cudaMalloc(&b->dwitems, sizeof(WItem) * nw);
            if (e == cudaSuccess) e = cudaMallocHost(&b->hwitems, sizeof(WItem) * nw);
        }
    }
    if (e != cudaSuccess) return bail(bcuda(nullptr, e, "lbm_batch_create allocation"));
    e = plan_grid(b);
    if (e != cudaSuccess) return bail(bcuda(nullptr, e, "lbm_batch_create occupancy"));
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    BGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->hist);
    cudaFree(b->dinst);
    cudaFree(b->ditems);
    cudaFree(b->dranges);
    cudaFree(b->dcounts);
    cudaFree(b->partials);
    cudaFree(b->dsums);
    cudaFree(b->fields);
    cudaFree(b->maxbits);
    cudaFreeHost(b->hsums);
    cudaFreeHost(b->hitems);
    cudaFreeHost(b->hranges);
    cudaFreeHost(b->hcounts);
    cudaFree(b->dwitems);
    cudaFreeHost(b->hwitems);
    delete b;
}

lbm_status lbm_batch_init(lbm_batch *b, const double *e, const double *qx, const double *qy) {
    NvtxRange nvtx_("lbm_batch_init");
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    BGuard g(b->device);
    drop_graph(b);
    // 16-bit storage: one power-of-two scale for all instances
    b->scale = 1.0;
    double amax = 0.0;
    long long base = 0;
    for (int i = 0; i < b->count; ++i) {
        const long long n = (long long)b->inst[i].nx * b->inst[i].ny;
        for (long long j = 0; j < n; ++j) {
            double v = e ? (2.0 / 9.0) * std::fabs(e[base + j] - b->e_ref) : 0.0;
            if (qx) v += std::fabs(qx[base + j]) / 3.0;
            if (qy) v += std::fabs(qy[base + j]) / 3.0;
            if (!std::isfinite(v)) return bfail(b, LBM_EINVAL, "initial fields are not finite");
            amax = std::fmax(amax, v);
        }
        amax = std::fmax(amax, (2.0 / 9.0) * std::fabs(b->inst[i].bc.delta_e));
        base += n;
    }
    if ((b->precision == PREC_FP16 || b->precision == PREC_BF16) && amax > 0.0) {
        int ex;
        std::frexp(amax, &ex);
        int p = 12 - ex;
        p = p > 100 ? 100 : (p < -100 ? -100 : p);
        b->scale = std::ldexp(1.0, p);
    }
    BCK(b, upload_table_any(b));
    base = 0;
    for (int i = 0; i < b->count; ++i) {
        const lbm_instance &in = b->inst[i];
        const long long n = (long long)in.nx * in.ny;
        double *de = b->fields, *dqx = b->fields + b->max_plane, *dqy = b->fields + 2 * b->max_plane;
        if (e) {
            BCK(b, cudaMemcpyAsync(de, e + base, sizeof(double) * n, cudaMemcpyHostToDevice,
                                   b->stream));
        } else {
            std::vector<double> flat(n, b->e_ref);
            BCK(b, cudaMemcpyAsync(de, flat.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                                   b->stream));
            BCK(b, cudaStreamSynchronize(b->stream));
        }
        if (qx)
            BCK(b, cudaMemcpyAsync(dqx, qx + base, sizeof(double) * n, cudaMemcpyHostToDevice,
                                   b->stream));
        if (qy)
            BCK(b, cudaMemcpyAsync(dqy, qy + base, sizeof(double) * n, cudaMemcpyHostToDevice,
                                   b->stream));
        cudaError_t err;
        const long long o = b->off[i];
        switch (b->precision) {
            case PREC_FP32:
                err = launch_init<float>(de, qx ? dqx : nullptr, qy ? dqy : nullptr, in.nx, in.ny,
                                         b->e_ref, b->scale, coef_of<float>(in, b->scale, b->precision),
                                         (float *)b->buf[1] + o, (float *)b->buf[0] + o,
                                         b->stream);
                break;
            case PREC_FP64:
                err = launch_init<double>(de, qx ? dqx : nullptr, qy ? dqy : nullptr, in.nx,
                                          in.ny, b->e_ref, b->scale,
                                          coef_of<double>(in, b->scale, b->precision),
                                          (double *)b->buf[1] + o, (double *)b->buf[0] + o,
                                          b->stream);
                break;
            case PREC_FP16:
                err = launch_init<__half>(de, qx ? dqx : nullptr, qy ? dqy : nullptr, in.nx,
                                          in.ny, b->e_ref, b->scale,
                                          coef_of<float>(in, b->scale, b->precision), (__half *)b->buf[1] + o,
                                          (__half *)b->buf[0] + o, b->stream);
                break;
            default:
                err = launch_init<__nv_bfloat16>(
                    de, qx ? dqx : nullptr, qy ? dqy : nullptr, in.nx, in.ny, b->e_ref, b->scale,
                    coef_of<float>(in, b->scale, b->precision), (__nv_bfloat16 *)b->buf[1] + o,
                    (__nv_bfloat16 *)b->buf[0] + o, b->stream);
        }
        if (err != cudaSuccess) return bcuda(b, err, "batch init kernel");
        BCK(b, cudaStreamSynchronize(b->stream));   // staging reused by the next instance
        base += n;
    }
    // no history yet: zero it so the first comparison reads defined values
    BCK(b, cudaMemsetAsync(b->hist, 0, csize(b->precision) * b->htotal, b->stream));
    b->cur = 0;
    b->initialised = true;
    b->have_prev = false;
    std::fill(b->active.begin(), b->active.end(), 1);
    std::fill(b->icur.begin(), b->icur.end(), 0);
    std::fill(b->steps.begin(), b->steps.end(), 0);
    std::fill(b->prev_step.begin(), b->prev_step.end(), 0);
    std::fill(b->good.begin(), b->good.end(), 0);
    std::fill(b->last_r.begin(), b->last_r.end(), INFINITY);
    BCK(b, rebuild_items(b));
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, long n) {
    NvtxRange nvtx_("lbm_batch_step");
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (n < 0) return bfail(b, LBM_EINVAL, "n must be >= 0");
    if (!b->initialised) return bfail(b, LBM_EINVAL, "lbm_batch_init has not been called");
    BGuard g(b->device);
    if (n > 0) {
        // the read-outs pull the state from the buffer the last step read,
        // which a multi-step launch does not leave: end with a single step
        BCK(b, plain_steps(b, n - 1, &b->cur, b->stream));
        BCK(b, launch_any(b, B_STEP, b->cur, b->stream));
        b->cur = 1 - b->cur;
    }
    for (int i = 0; i < b->count; ++i)
        if (b->active[i]) {
            b->steps[i] += n;
            b->icur[i] = b->cur;
        }
    return LBM_OK;
}

lbm_status lbm_batch_residuals(lbm_batch *b, double *r, double *energy) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!b->initialised) return bfail(b, LBM_EINVAL, "lbm_batch_init has not been called");
    BGuard g(b->device);
    bool any_zero = false;
    for (int i = 0; i < b->count; ++i) any_zero |= b->active[i] && b->steps[i] == 0;
    if (any_zero)
        return bfail(b, LBM_EUNSUPPORTED, "residuals need at least one step since init");
    // read-only pass over the state of every active instance (pulled from
    // the buffer read last)
    BCK(b, launch_any(b, B_RES_ONLY, 1 - b->cur, b->stream));
    BCK(b, launch_finalize_batch(b, b->stream));
    BCK(b, cudaMemcpyAsync(b->hsums, b->dsums, sizeof(double) * 5 * b->count,
                           cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    bool bad = false;
    for (int i = 0; i < b->count; ++i) {
        if (!b->active[i]) continue;
        const double *s = b->hsums + 5 * i;
        finish(b, i, s, nullptr);
        const double n = (double)b->inst[i].nx * b->inst[i].ny;
        if (energy) energy[i] = n * b->e_ref + s[0];
        bad |= s[4] > 0.0;
    }
    b->have_prev = true;
    if (r)
        for (int i = 0; i < b->count; ++i) r[i] = b->last_r[i];
    if (bad) return bfail(b, LBM_ENONFINITE, "an instance holds NaN or Inf");
    return LBM_OK;
}

lbm_status lbm_batch_solve(lbm_batch *b, double tol, int check_every, long max_steps,
                           long *steps, double *r) {
    NvtxRange nvtx_("lbm_batch_solve");
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!b->initialised) return bfail(b, LBM_EINVAL, "lbm_batch_init has not been called");
    if (!(tol > 0.0)) return bfail(b, LBM_EINVAL, "tol must be > 0");
    if (check_every < 2 || (check_every & 1))
        return bfail(b, LBM_EINVAL, "check_every must be an even number >= 2");
    if (max_steps < 0) return bfail(b, LBM_EINVAL, "max_steps must be >= 0");
    BGuard g(b->device);
    // one captured graph per starting buffer: check_every - 1 plain steps
    // (multi-step launches when set), then the step with the residual sums
    if (b->graph_k != check_every) drop_graph(b);
    const long window_launches = plain_launches(b, check_every - 1) + 1;
    for (int start = 0; start < 2; ++start) {
        if (b->graph[start]) continue;
        cudaStream_t cap = nullptr;
        BCK(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int src = start;
        if (e == cudaSuccess) e = plain_steps(b, check_every - 1, &src, cap);
        // have_prev is a launch argument: capture the comparing variant;
        // the first window's comparison is ignored (no history yet)
        const bool hp = b->have_prev;
        b->have_prev = true;
        if (e == cudaSuccess) e = launch_any(b, B_STEP_RES, src, cap);
        b->have_prev = hp;
        if (e == cudaSuccess) e = launch_finalize_batch(b, cap);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->hsums, b->dsums, sizeof(double) * 5 * b->count,
                                cudaMemcpyDeviceToHost, cap);
        cudaGraph_t gr = nullptr;
        cudaError_t ee = cudaStreamEndCapture(cap, &gr);
        cudaStreamDestroy(cap);
        if (e == cudaSuccess) e = ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[start], gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            b->graph[start] = nullptr;
            return bcuda(b, e, "batch window capture");
        }
        b->graph_k = check_every;
    }

    bool bad = false;
    while (true) {
        bool any = false;
        for (int i = 0; i < b->count; ++i) any |= b->active[i] && b->steps[i] < max_steps;
        if (!any) break;
        // instances that reached max_steps stop too
        bool changed = false;
        for (int i = 0; i < b->count; ++i)
            if (b->active[i] && b->steps[i] >= max_steps) {
                b->active[i] = 0;
                changed = true;
            }
        if (changed) BCK(b, rebuild_items(b));
        BCK(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        if (window_launches & 1) b->cur = 1 - b->cur;
        changed = false;
        for (int i = 0; i < b->count; ++i) {
            if (!b->active[i]) continue;
            b->steps[i] += check_every;
            b->icur[i] = b->cur;
            double ri;
            finish(b, i, b->hsums + 5 * i, &ri);
            if (std::isnan(ri)) {
                bad = true;
                b->active[i] = 0;
                changed = true;
                continue;
            }
            b->good[i] = b->last_r[i] < tol ? b->good[i] + 1 : 0;
            if (b->good[i] >= 2) {
                b->active[i] = 0;          // steady: retire
                changed = true;
            }
        }
        b->have_prev = true;
        if (changed) BCK(b, rebuild_items(b));
    }
    for (int i = 0; i < b->count; ++i) {
        if (steps) steps[i] = b->steps[i];
        if (r) r[i] = b->last_r[i];
    }
    if (bad) return bfail(b, LBM_ENONFINITE, "an instance became non-finite (retired)");
    return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch *b, int i, double *e, double *qx, double *qy) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->count) return bfail(b, LBM_EINVAL, "instance index out of range");
    if (!b->initialised) return bfail(b, LBM_EINVAL, "lbm_batch_init has not been called");
    BGuard g(b->device);
    const lbm_instance &in = b->inst[i];
    const long long n = (long long)in.nx * in.ny;
    const Params p = params_of(in);
    Readout rd;
    rd.nx = in.nx;
    rd.ny = in.ny;
    rd.bc_x = in.bc.x;
    rd.bc_y = in.bc.y;
    rd.pulled = b->steps[i] > 0;
    rd.e_ref = b->e_ref;
    rd.inv_scale = 1.0 / b->scale;
    rd.kappa = p.kappa;
    double *d[3] = {b->fields, b->fields + b->max_plane, b->fields + 2 * b->max_plane};
    const long long o = b->off[i];
    const int src = 1 - b->icur[i];      // the buffer this instance read last
    cudaError_t err;
    switch (b->precision) {
        case PREC_FP32:
            err = launch_moments<float>((const float *)b->buf[src] + o, rd,
                                        coef_of<float>(in, b->scale, b->precision), d[0], d[1], d[2],
                                        b->stream);
            break;
        case PREC_FP64:
            err = launch_moments<double>((const double *)b->buf[src] + o, rd,
                                         coef_of<double>(in, b->scale, b->precision), d[0], d[1], d[2],
                                         b->stream);
            break;
        case PREC_FP16:
            err = launch_moments<__half>((const __half *)b->buf[src] + o, rd,
                                         coef_of<float>(in, b->scale, b->precision), d[0], d[1], d[2],
                                         b->stream);
            break;
        default:
            err = launch_moments<__nv_bfloat16>((const __nv_bfloat16 *)b->buf[src] + o, rd,
                                                coef_of<float>(in, b->scale, b->precision), d[0], d[1], d[2],
                                                b->stream);
    }
    if (err != cudaSuccess) return bcuda(b, err, "batch moments");
    double *h[3] = {e, qx, qy};
    for (int f = 0; f < 3; ++f)
        if (h[f])
            BCK(b, cudaMemcpyAsync(h[f], d[f], sizeof(double) * n, cudaMemcpyDeviceToHost,
                                   b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

lbm_status lbm_batch_set_schedule(lbm_batch *b, int threads_per_item, int ctas_per_sm) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (threads_per_item != 128 && threads_per_item != 256 && threads_per_item != 512)
        return bfail(b, LBM_EINVAL, "threads_per_item must be 128, 256 or 512");
    if (ctas_per_sm < 0) return bfail(b, LBM_EINVAL, "ctas_per_sm must be >= 0");
    BGuard g(b->device);
    const int old_t = b->tpi, old_c = b->ctas_per_sm;
    b->tpi = threads_per_item;
    b->ctas_per_sm = ctas_per_sm;
    cudaError_t e = plan_grid(b);
    if (e != cudaSuccess) {
        b->tpi = old_t;
        b->ctas_per_sm = old_c;
        plan_grid(b);
        return bcuda(b, e, "batch schedule");
    }
    drop_graph(b);
    if (b->initialised) BCK(b, rebuild_items(b));
    return LBM_OK;
}

lbm_status lbm_batch_get_schedule(const lbm_batch *b, int *threads_per_item, int *ctas_per_sm,
                                  int *grid) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (threads_per_item) *threads_per_item = b->tpi;
    if (ctas_per_sm) *ctas_per_sm = b->grid / (b->sms > 0 ? b->sms : 1);
    if (grid) *grid = b->grid;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int trial_steps, double *us_per_step) {
    NvtxRange nvtx_("lbm_batch_autotune");
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!b->initialised) return bfail(b, LBM_EINVAL, "lbm_batch_init has not been called");
    if (trial_steps < 0) return bfail(b, LBM_EINVAL, "trial_steps must be >= 0");
    if (trial_steps == 0) trial_steps = 10;
    if (trial_steps & 1) ++trial_steps;
    BGuard g(b->device);
    // timings run on the live buffers: keep a copy of the state
    const size_t bytes = elem_size(b->precision) * b->total;
    void *saved = nullptr;
    BCK(b, cudaMallocAsync(&saved, 2 * bytes, b->stream));
    for (int i = 0; i < 2; ++i)
        BCK(b, cudaMemcpyAsync((char *)saved + i * bytes, b->buf[i], bytes,
                               cudaMemcpyDeviceToDevice, b->stream));
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    const int old_t = b->tpi, old_c = b->ctas_per_sm;
    float best = -1.f;
    int best_t = old_t, best_c = old_c;
    cudaError_t err = cudaSuccess;
    for (int tpi : {128, 256, 512}) {
        for (int cps : {0, 1, 2}) {
            b->tpi = tpi;
            b->ctas_per_sm = cps;
            if (plan_grid(b) != cudaSuccess) {
                (void)cudaGetLastError();
                continue;
            }
            if ((err = rebuild_items(b)) != cudaSuccess) break;
            for (int s = 0; s < 2 && err == cudaSuccess; ++s)
                err = launch_any(b, B_STEP, s & 1, b->stream);
            if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
            for (int s = 0; s < trial_steps && err == cudaSuccess; ++s)
                err = launch_any(b, B_STEP, s & 1, b->stream);
            if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) break;
            if (best < 0.f || ms < best) {
                best = ms;
                best_t = tpi;
                best_c = cps;
            }
        }
        if (err != cudaSuccess) break;
    }
    // multi-step launches (FP32): per-step time of launches of K steps with
    // the best single-step schedule for the other launches
    const int old_ws = b->wave_steps, old_wr = b->wave_rows;
    int best_ws = 0, best_wr = old_wr;
    float best_step = best / trial_steps;      // ms per step of the single steps
    if (err == cudaSuccess && b->precision == PREC_FP32 && b->dwitems) {
        b->tpi = best_t;
        b->ctas_per_sm = best_c;
        if (plan_grid(b) != cudaSuccess) (void)cudaGetLastError();
        for (int ks : {3, 4, 5}) {
            for (int rows : {64, 128}) {
                b->wave_steps = ks;
                b->wave_rows = rows;
                if ((err = rebuild_items(b)) != cudaSuccess) break;
                const int launches = 2 * ((trial_steps + 2 * ks - 1) / (2 * ks));
                for (int s = 0; s < 2 && err == cudaSuccess; ++s)
                    err = launch_wave(b, ks, s & 1, b->stream);
                if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
                for (int s = 0; s < launches && err == cudaSuccess; ++s)
                    err = launch_wave(b, ks, s & 1, b->stream);
                if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (err != cudaSuccess) break;
                const float per_step = ms / (launches * ks);
                if (per_step < best_step) {
                    best_step = per_step;
                    best_ws = ks;
                    best_wr = rows;
                }
            }
            if (err != cudaSuccess) break;
        }
    }
    b->wave_steps = err == cudaSuccess ? best_ws : old_ws;
    b->wave_rows = err == cudaSuccess ? best_wr : old_wr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < 2 && err == cudaSuccess; ++i)
        err = cudaMemcpyAsync(b->buf[i], (char *)saved + i * bytes, bytes,
                              cudaMemcpyDeviceToDevice, b->stream);
    cudaFreeAsync(saved, b->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
    b->tpi = best_t;
    b->ctas_per_sm = best_c;
    cudaError_t pe = plan_grid(b);
    drop_graph(b);
    if (err == cudaSuccess) err = pe;
    if (err == cudaSuccess) err = rebuild_items(b);
    if (err != cudaSuccess) return bcuda(b, err, "lbm_batch_autotune");
    if (us_per_step) *us_per_step = best >= 0.f ? 1000.0 * best_step : 0.0;
    return LBM_OK;
}

lbm_status lbm_batch_set_wave(lbm_batch *b, int steps, int rows) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (steps != 0 && (steps < WAVE_MIN_STEPS || steps > WAVE_MAX_STEPS))
        return bfail(b, LBM_EINVAL, "steps per launch must be 0 or 2..8");
    if (rows < 1) return bfail(b, LBM_EINVAL, "rows per segment must be >= 1");
    if (steps && b->precision != PREC_FP32)
        return bfail(b, LBM_EUNSUPPORTED, "multi-step launches need LBM_FP32 storage");
    if (steps) {
        for (int i = 0; i < b->count; ++i)
            if (b->inst[i].nx % 2)
                return bfail(b, LBM_EUNSUPPORTED, "multi-step launches need even nx");
    }
    BGuard g(b->device);
    b->wave_steps = steps;
    b->wave_rows = rows;
    drop_graph(b);
    if (b->initialised) BCK(b, rebuild_items(b));
    return LBM_OK;
}

lbm_status lbm_batch_get_wave(const lbm_batch *b, int *steps, int *rows) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (steps) *steps = b->wave_steps;
    if (rows) *rows = b->wave_rows;
    return LBM_OK;
}

long lbm_batch_active(const lbm_batch *b) {
    if (!b) return -1;
    long n = 0;
    for (char a : b->active) n += a ? 1 : 0;
    return n;
}

long lbm_batch_steps(const lbm_batch *b, int i) {
    if (!b || i < 0 || i >= b->count) return -1;
    return b->steps[i];
}

// Heat-flux unit of a channel's normalised profile: (5/9) tau_R delta_e / nx,
// i.e. the Fourier flux (1/3) C_V v_g^2 tau_R |dT/dx| in lattice units with
// the steady slope |de/dx| = delta_e / nx of Eqs. 59-60.
static double q_unit_of(const lbm_instance &in) {
    return (5.0 / 9.0) * in.tau_R * in.bc.delta_e / in.nx;
}

static bool profile_ok(const lbm_instance &in) {
    return in.bc.x == LBM_BC_PERIODIC_GRADIENT && in.bc.delta_e != 0.0 &&
           std::isfinite(in.tau_R);
}

lbm_status lbm_batch_profiles(lbm_batch *b, float *out) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!out) return bfail(b, LBM_EINVAL, "out is NULL");
    if (!b->initialised) return bfail(b, LBM_EINVAL, "lbm_batch_init has not been called");
    for (int i = 0; i < b->count; ++i)
        if (!profile_ok(b->inst[i]))
            return bfail(b, LBM_EUNSUPPORTED,
                         "instance " + std::to_string(i) +
                             ": profiles need the periodic temperature gradient (delta_e != 0) "
                             "and finite tau_R");
    BGuard g(b->device);
    for (int i = 0; i < b->count; ++i) {
        const lbm_instance &in = b->inst[i];
        const Params p = params_of(in);
        Readout rd;
        rd.nx = in.nx;
        rd.ny = in.ny;
        rd.bc_x = in.bc.x;
        rd.bc_y = in.bc.y;
        rd.pulled = b->steps[i] > 0;
        rd.e_ref = b->e_ref;
        rd.inv_scale = 1.0 / b->scale;
        rd.kappa = p.kappa;
        double *d[3] = {b->fields, b->fields + b->max_plane, b->fields + 2 * b->max_plane};
        const long long o = b->off[i];
        const int src = 1 - b->icur[i];
        cudaError_t err;
        switch (b->precision) {
            case PREC_FP32:
                err = launch_moments<float>((const float *)b->buf[src] + o, rd,
                                            coef_of<float>(in, b->scale, b->precision), d[0], d[1], nullptr,
                                            b->stream);
                break;
            case PREC_FP64:
                err = launch_moments<double>((const double *)b->buf[src] + o, rd,
                                             coef_of<double>(in, b->scale, b->precision), d[0], d[1], nullptr,
                                             b->stream);
                break;
            case PREC_FP16:
                err = launch_moments<__half>((const __half *)b->buf[src] + o, rd,
                                             coef_of<float>(in, b->scale, b->precision), d[0], d[1], nullptr,
                                             b->stream);
                break;
            default:
                err = launch_moments<__nv_bfloat16>((const __nv_bfloat16 *)b->buf[src] + o, rd,
                                                    coef_of<float>(in, b->scale, b->precision), d[0], d[1],
                                                    nullptr, b->stream);
        }
        if (err != cudaSuccess) return bcuda(b, err, "batch profile moments");
        channel_profile<<<PROFILE_POINTS, 128, 0, b->stream>>>(
            d[0], d[1], in.nx, in.ny, b->e_ref, in.bc.delta_e, q_unit_of(in),
            out + (size_t)i * 2 * PROFILE_POINTS);
        BCK(b, cudaGetLastError());
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// Eq. 68: the heat flux across a channel of width d between diffuse walls
// under a uniform temperature gradient, over the Fourier flux, from the
// phonon hydrodynamic model with the slip condition of Eq. 11, at Y = y/d:
//   Q(Y) = 1 - (exp((Y - 1)/Kn_eff) + exp(-Y/Kn_eff)) /
//              (1 + exp(-1/Kn_eff) + (8/15)(Kn_C/Kn_eff)(1 - exp(-1/Kn_eff))),
// Kn_eff = sqrt(tau_C tau_R v_g^2 / 5) / d, Kn_C = v_g tau_C / d.  In lattice
// units v_g = sqrt(5/3) and tau_C = 1 / (1/tau_N + 1/tau_R) (Section 2.1).
static double eq68_flux(double Y, double tau_N, double tau_R, double d) {
    const double tau_C = 1.0 / ((std::isinf(tau_N) ? 0.0 : 1.0 / tau_N) + 1.0 / tau_R);
    const double vg2 = 5.0 / 3.0;
    const double kn_eff = std::sqrt(tau_C * tau_R * vg2 / 5.0) / d;
    const double kn_c = std::sqrt(vg2) * tau_C / d;
    const double a = std::exp(-1.0 / kn_eff);
    const double num = std::exp((Y - 1.0) / kn_eff) + std::exp(-Y / kn_eff);
    const double den = 1.0 + a + (8.0 / 15.0) * (kn_c / kn_eff) * (1.0 - a);
    return 1.0 - num / den;
}

lbm_status lbm_analytic_profiles(const lbm_instance *inst, int count, float *out, int op,
                                 void *stream) {
    if (!inst || !out || count < 1) return bfail(nullptr, LBM_EINVAL, "bad arguments");
    if (op < -1 || op > 1) return bfail(nullptr, LBM_EINVAL, "op must be -1, 0 or 1");
    for (int i = 0; i < count; ++i) {
        const lbm_instance &in = inst[i];
        if (in.bc.y != LBM_BC_DIFFUSE_WALLS || in.ny < 2 || !std::isfinite(in.tau_R) ||
            !(in.tau_R > 0.0) || !(in.tau_N > 0.0))
            return bfail(nullptr, LBM_EUNSUPPORTED,
                         "instance " + std::to_string(i) +
                             ": the analytic profile needs walls on y, ny >= 2 and finite "
                             "tau_R");
    }
    std::vector<float> prof((size_t)count * 2 * PROFILE_POINTS, 0.f);
    for (int i = 0; i < count; ++i) {
        const lbm_instance &in = inst[i];
        const double d = in.ny - 1;       // the walls sit on rows 0 and ny - 1
        float *p = prof.data() + (size_t)i * 2 * PROFILE_POINTS;
        for (int j = 0; j < PROFILE_POINTS; ++j)
            p[j] = (float)eq68_flux((double)j / (PROFILE_POINTS - 1), in.tau_N, in.tau_R, d);
        // E(Y) = 0: e affine in x with the steady slope, uniform across
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = prof.size();
    cudaError_t e = cudaSuccess;
    if (op == 0) {
        e = cudaMemcpyAsync(out, prof.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
    } else {
        float *tmp = nullptr;
        e = cudaMalloc(&tmp, sizeof(float) * n);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp, prof.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            add_scaled<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, tmp, (float)op,
                                                                  (long long)n);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(tmp);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(nullptr, e, "lbm_analytic_profiles");
    return LBM_OK;
}

lbm_status lbm_batch_init_profiles(lbm_batch *b, const float *profiles) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (!profiles) return bfail(b, LBM_EINVAL, "profiles is NULL");
    if (b->precision == PREC_FP16 || b->precision == PREC_BF16)
        return bfail(b, LBM_EUNSUPPORTED, "profile start needs FP32 or FP64 storage");
    for (int i = 0; i < b->count; ++i)
        if (!profile_ok(b->inst[i]))
            return bfail(b, LBM_EUNSUPPORTED, "instance " + std::to_string(i) +
                                                  ": profiles need the periodic temperature "
                                                  "gradient and finite tau_R");
    BGuard g(b->device);
    drop_graph(b);
    b->scale = 1.0;
    BCK(b, upload_table_any(b));
    for (int i = 0; i < b->count; ++i) {
        const lbm_instance &in = b->inst[i];
        const long long n = (long long)in.nx * in.ny;
        double *de = b->fields, *dqx = b->fields + b->max_plane, *dqy = b->fields + 2 * b->max_plane;
        long long blocks = (n + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        const float *prof = profiles + (size_t)i * 2 * PROFILE_POINTS;
        double *emean = b->dsums + 5 * i;      // scratch slot of this instance
        profile_e_mean<<<1, 128, 0, b->stream>>>(prof, in.ny, emean);
        BCK(b, cudaGetLastError());
        channel_fields<<<(unsigned)blocks, 256, 0, b->stream>>>(
            prof, in.nx, in.ny, b->e_ref, in.bc.delta_e, q_unit_of(in), emean, de, dqx, dqy);
        BCK(b, cudaGetLastError());
        const long long o = b->off[i];
        cudaError_t err;
        if (b->precision == PREC_FP32)
            err = launch_init<float>(de, dqx, dqy, in.nx, in.ny, b->e_ref, 1.0,
                                     coef_of<float>(in, 1.0, b->precision), (float *)b->buf[1] + o,
                                     (float *)b->buf[0] + o, b->stream);
        else
            err = launch_init<double>(de, dqx, dqy, in.nx, in.ny, b->e_ref, 1.0,
                                      coef_of<double>(in, 1.0, b->precision), (double *)b->buf[1] + o,
                                      (double *)b->buf[0] + o, b->stream);
        if (err != cudaSuccess) return bcuda(b, err, "batch profile init");
    }
    BCK(b, cudaMemsetAsync(b->hist, 0, csize(b->precision) * b->htotal, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->cur = 0;
    b->initialised = true;
    b->have_prev = false;
    std::fill(b->active.begin(), b->active.end(), 1);
    std::fill(b->icur.begin(), b->icur.end(), 0);
    std::fill(b->steps.begin(), b->steps.end(), 0);
    std::fill(b->prev_step.begin(), b->prev_step.end(), 0);
    std::fill(b->good.begin(), b->good.end(), 0);
    std::fill(b->last_r.begin(), b->last_r.end(), INFINITY);
    BCK(b, rebuild_items(b));
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) {
    if (!b) return "batch is NULL";
    return b->err.c_str();
}

}  // extern "C"
