// The phonon lattice Boltzmann step on the one-dimensional D1Q2 and the
// three-dimensional D3Q14 lattices (Section 2.2 names both; their weights
// follow from the moment conditions of Section 2.3, see phonon_lbm.h), on
// periodic lattices, behind the lbm_nd_* entry points.
//
// Same design as the D2Q8 path: structure of arrays (Q planes of
// nx*ny*nz, x fastest), deviations d_i = s (e_i - w_i e_ref) with s = 1,
// pull streaming from the post-collision planes of the previous step, the
// collision in registers on deviations with exact-sum rounded weights, and
// captured CUDA graphs of 64 steps.  In a pull step every stored value is
// read by exactly one node, so one thread per node with x fastest reads each
// plane row once, coalesced (the +-1 shift along x costs one extra sector
// per warp, served from L2).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/phonon_lbm.h"
#include "lbm_kernels.h"

namespace plbm {
namespace {

// Velocity sets, with opposite velocities at adjacent indices (2j, 2j+1).
// D3Q14: i = 0..5 the axis velocities +x, -x, +y, -y, +z, -z; i = 6..13
// the corners +b_j, -b_j for b_j = (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1).
// D1Q2: +x, -x.
template <int LAT> struct Lat;
template <> struct Lat<LBM_LATTICE_D3Q14> {
    static constexpr int Q = 14, DIM = 3, AXIS = 6;
    __host__ __device__ static constexpr int sgn(int i) { return (i & 1) ? -1 : 1; }
    __host__ __device__ static constexpr int cx(int i) {
        return i < 6 ? (i < 2 ? sgn(i) : 0) : sgn(i);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return i < 6 ? (i == 2 || i == 3 ? sgn(i) : 0) : sgn(i) * ((((i - 6) >> 2) & 1) ? -1 : 1);
    }
    __host__ __device__ static constexpr int cz(int i) {
        return i < 6 ? (i >= 4 ? sgn(i) : 0) : sgn(i) * ((((i - 6) >> 1) & 1) ? -1 : 1);
    }
};
template <> struct Lat<LBM_LATTICE_D1Q2> {
    static constexpr int Q = 2, DIM = 1, AXIS = 2;
    __host__ __device__ static constexpr int cx(int i) { return i == 0 ? 1 : -1; }
    __host__ __device__ static constexpr int cy(int) { return 0; }
    __host__ __device__ static constexpr int cz(int) { return 0; }
};

// Coefficients rounded once to the compute type C.  Eq. 13 on deviations:
// rho = sum d_i, m = sum c_i d_i, q = m - lambda m (Eq. 54), t_i = h_i c_i.q,
// eq_i = w_i rho + t_i (Eq. 15), d_i* = d_i - omega (d_i - eq_i) - sigma t_i
// (Eq. 16).  The rounded weights keep sum_i w_i = 1 and sum_i h_i c_ix^2 = 1
// exact (see exact_pair), so the collision conserves energy and, without
// resistive scattering, heat flux to rounding.
template <typename C> struct CoefN {
    C omega, sigma, lambda;
    C w_axis, w_corner;
    C h_axis, h_corner;
};

// The collision of one node, on Q pulled deviations.
template <int LAT, typename C>
__device__ __forceinline__ void collide_nd(C (&d)[Lat<LAT>::Q], const CoefN<C> &k) {
    using L = Lat<LAT>;
    C rho = C(0), mx = C(0), my = C(0), mz = C(0);
#pragma unroll
    for (int i = 0; i < L::Q; i += 2) {       // opposite velocities are adjacent
        rho += d[i] + d[i + 1];
        if (L::cx(i)) mx += L::cx(i) > 0 ? d[i] - d[i + 1] : d[i + 1] - d[i];
        if (L::cy(i)) my += L::cy(i) > 0 ? d[i] - d[i + 1] : d[i + 1] - d[i];
        if (L::cz(i)) mz += L::cz(i) > 0 ? d[i] - d[i + 1] : d[i + 1] - d[i];
    }
    const C qx = mx - k.lambda * mx, qy = my - k.lambda * my, qz = mz - k.lambda * mz;
    const C wa = k.w_axis * rho, wc = k.w_corner * rho;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        C cq = C(0);
        if (L::cx(i)) cq += L::cx(i) > 0 ? qx : -qx;
        if (L::cy(i)) cq += L::cy(i) > 0 ? qy : -qy;
        if (L::cz(i)) cq += L::cz(i) > 0 ? qz : -qz;
        const C t = (i < L::AXIS ? k.h_axis : k.h_corner) * cq;
        const C eq = (i < L::AXIS ? wa : wc) + t;
        d[i] = d[i] - k.omega * (d[i] - eq) - k.sigma * t;
    }
}

struct Dims {
    int nx, ny, nz;
    long long plane;
};

// Pull of the Q populations arriving at node (x, y, z) from the
// post-collision planes `src` of a periodic lattice.
template <int LAT, typename T>
__device__ __forceinline__ void pull_nd(const T *__restrict__ src, const Dims &g, int x, int y,
                                        int z, typename Store<T>::C (&d)[Lat<LAT>::Q]) {
    using L = Lat<LAT>;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int sx = x - L::cx(i), sy = y - L::cy(i), sz = z - L::cz(i);
        sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
        sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
        sz = sz < 0 ? sz + g.nz : (sz >= g.nz ? sz - g.nz : sz);
        d[i] = Store<T>::load(src[(long long)i * g.plane + ((long long)sz * g.ny + sy) * g.nx + sx]);
    }
}

template <int LAT, typename T>
__global__ void __launch_bounds__(256)
step_nd(const T *__restrict__ src, T *__restrict__ dst, Dims g, CoefN<typename Store<T>::C> k) {
    using C = typename Store<T>::C;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= g.plane) return;
    const int x = int(node % g.nx);
    const long long r = node / g.nx;
    const int y = int(r % g.ny), z = int(r / g.ny);
    C d[Lat<LAT>::Q];
    pull_nd<LAT, T>(src, g, x, y, z, d);
    collide_nd<LAT>(d, k);
#pragma unroll
    for (int i = 0; i < Lat<LAT>::Q; ++i) __stcs(dst + (long long)i * g.plane + node, Store<T>::put(d[i]));
}

// e and q of the state at the current step (pulled when `pulled`, else the
// stored step-0 state), FP64 outputs e[n], q[dim][n].
template <int LAT, typename T>
__global__ void moments_nd(const T *__restrict__ src, Dims g, bool pulled, double e_ref,
                           double inv_s, CoefN<typename Store<T>::C> k, double *e, double *q) {
    using C = typename Store<T>::C;
    using L = Lat<LAT>;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < g.plane;
         node += (long long)gridDim.x * blockDim.x) {
        const int x = int(node % g.nx);
        const long long r = node / g.nx;
        const int y = int(r % g.ny), z = int(r / g.ny);
        C d[L::Q];
        if (pulled) pull_nd<LAT, T>(src, g, x, y, z, d);
        else
#pragma unroll
            for (int i = 0; i < L::Q; ++i) d[i] = Store<T>::load(src[(long long)i * g.plane + node]);
        C rho = C(0), m[3] = {C(0), C(0), C(0)};
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            rho += d[i];
            m[0] += C(L::cx(i)) * d[i];
            m[1] += C(L::cy(i)) * d[i];
            m[2] += C(L::cz(i)) * d[i];
        }
        if (e) e[node] = e_ref + (double)rho * inv_s;
        if (q)
            for (int a = 0; a < L::DIM; ++a)
                q[(long long)a * g.plane + node] = (double)(m[a] - k.lambda * m[a]) * inv_s;
    }
}

template <int LAT, typename T>
__global__ void populations_nd(const T *__restrict__ src, Dims g, bool pulled, double e_ref,
                               double inv_s, double w_axis, double w_corner, double *f) {
    using C = typename Store<T>::C;
    using L = Lat<LAT>;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < g.plane;
         node += (long long)gridDim.x * blockDim.x) {
        const int x = int(node % g.nx);
        const long long r = node / g.nx;
        const int y = int(r % g.ny), z = int(r / g.ny);
        C d[L::Q];
        if (pulled) pull_nd<LAT, T>(src, g, x, y, z, d);
        else
#pragma unroll
            for (int i = 0; i < L::Q; ++i) d[i] = Store<T>::load(src[(long long)i * g.plane + node]);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            f[(long long)i * g.plane + node] =
                (double)d[i] * inv_s + (i < L::AXIS ? w_axis : w_corner) * e_ref;
    }
}

// Eq. 15 on deviations (compute type) as the step-0 state `pre`, and its
// collision as `post`.  e[n], q[dim][n] FP64 device arrays (q may be null).
template <int LAT, typename T>
__global__ void init_nd(const double *__restrict__ e, const double *__restrict__ q, Dims g,
                        double e_ref, CoefN<typename Store<T>::C> k, T *__restrict__ pre,
                        T *__restrict__ post) {
    using C = typename Store<T>::C;
    using L = Lat<LAT>;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < g.plane;
         node += (long long)gridDim.x * blockDim.x) {
        const C de = (C)(e[node] - e_ref);
        C qa[3] = {C(0), C(0), C(0)};
        if (q)
            for (int a = 0; a < L::DIM; ++a) qa[a] = (C)q[(long long)a * g.plane + node];
        C d[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const C cq = C(L::cx(i)) * qa[0] + C(L::cy(i)) * qa[1] + C(L::cz(i)) * qa[2];
            const C v = (i < L::AXIS ? k.w_axis : k.w_corner) * de +
                        (i < L::AXIS ? k.h_axis : k.h_corner) * cq;
            const T s = Store<T>::put(v);
            pre[(long long)i * g.plane + node] = s;
            d[i] = Store<T>::load(s);
        }
        collide_nd<LAT>(d, k);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) post[(long long)i * g.plane + node] = Store<T>::put(d[i]);
    }
}

// Per-block sums of (e - e_ref) and a non-finite count of the current state.
template <int LAT, typename T>
__global__ void __launch_bounds__(256)
energy_nd(const T *__restrict__ src, Dims g, bool pulled, double *__restrict__ partials) {
    using C = typename Store<T>::C;
    using L = Lat<LAT>;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < g.plane;
         base += stride) {
        const long long node = base + (threadIdx.x & 31);
        C loc[5] = {C(0), C(0), C(0), C(0), C(0)};
        if (node < g.plane) {
            const int x = int(node % g.nx);
            const long long r = node / g.nx;
            const int y = int(r % g.ny), z = int(r / g.ny);
            C d[L::Q];
            if (pulled) pull_nd<LAT, T>(src, g, x, y, z, d);
            else
#pragma unroll
                for (int i = 0; i < L::Q; ++i)
                    d[i] = Store<T>::load(src[(long long)i * g.plane + node]);
            C rho = C(0);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) rho += d[i];
            loc[0] = rho;
            loc[4] = isfinite(rho) ? C(0) : C(1);
        }
        warp_flush_residual(loc, acc);
    }
    block_sum5_lane0(acc, partials + (size_t)blockIdx.x * 5);
}

constexpr int ENERGY_BLOCKS = 1216;

unsigned grid_of(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    return (unsigned)(b > 0 ? b : 1);
}

// Rounds w_a (count na) and w_c (count nc) to C so that na w_a + nc w_c == 1
// holds exactly in C's binary arithmetic: start from the nearest value of
// the exact w_a and step one unit in the last place at a time until the
// w_c it implies is exactly representable.  For double nothing is checked
// (rounding there moves the sum by ~1e-16 per step).
template <typename C> void exact_pair(double wa, int na, int nc, C &oa, C &oc);
template <> void exact_pair<double>(double wa, int na, int nc, double &oa, double &oc) {
    oa = wa;
    oc = (1.0 - na * wa) / nc;
}
template <> void exact_pair<float>(double wa, int na, int nc, float &oa, float &oc) {
    float a = (float)wa;
    for (int k = 0; k < 64; ++k) {
        for (int sgn = 0; sgn < 2; ++sgn) {
            float t = a;
            for (int s = 0; s < k; ++s) t = std::nextafter(t, sgn ? 1.0f : 0.0f);
            const double rest = 1.0 - na * (double)t;   // exact: float times small int
            const float c = (float)(rest / nc);
            if ((double)c * nc == rest) {                // exact in double for floats
                oa = t;
                oc = c;
                return;
            }
        }
    }
    oa = a;
    oc = (float)((1.0 - na * wa) / nc);
}

}  // namespace
}  // namespace plbm

using namespace plbm;

struct lbm_nd {
    int lattice = 0, dim = 0, Q = 0;
    int precision = 0;
    int device = 0;
    Dims g{};
    double tau_N = 0, tau_R = 0, tau = 0, tau_r = 0, kappa = 1, sigma = 0;
    double e_ref = 1.0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    void *buf[2] = {nullptr, nullptr};
    size_t buf_bytes = 0;
    int cur = 0;
    long n = 0;
    bool initialised = false;
    double *fields = nullptr;       // (1 + dim) planes of doubles
    double *partials = nullptr;     // ENERGY_BLOCKS x 5
    double *sums = nullptr;         // 5
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_chunk = 64;
    std::string err;
};

namespace {

thread_local std::string g_nd_error;

lbm_status nd_fail(lbm_nd *c, lbm_status s, const std::string &m) {
    if (c) c->err = m;
    else g_nd_error = m;
    return s;
}

lbm_status nd_cuda(lbm_nd *c, cudaError_t e, const char *where) {
    (void)cudaGetLastError();
    return nd_fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

#define NDCK(c, call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return nd_cuda(c, e_, #call);   \
    } while (0)

template <typename C> CoefN<C> coef_nd(const lbm_nd *c) {
    CoefN<C> k{};
    k.omega = (C)(1.0 / c->tau);
    k.sigma = (C)c->sigma;
    k.lambda = (C)(std::isinf(c->tau_r) ? 0.0 : 1.0 / (2.0 * c->tau_r + 1.0));
    if (c->lattice == LBM_LATTICE_D3Q14) {
        exact_pair<C>(1.0 / 9.0, 6, 8, k.w_axis, k.w_corner);    // 6 w_a + 8 w_c = 1
        exact_pair<C>(1.0 / 3.0, 2, 8, k.h_axis, k.h_corner);    // 2 h_a + 8 h_c = 1
    } else {
        k.w_axis = k.w_corner = (C)0.5;
        k.h_axis = k.h_corner = (C)0.5;
    }
    return k;
}

// Calls F<LAT, T>::run(c, args...) for the context's lattice and storage.
template <template <int, typename> class F, typename... A>
cudaError_t nd_dispatch(const lbm_nd *c, A... a) {
    if (c->lattice == LBM_LATTICE_D3Q14) {
        if (c->precision == PREC_FP64) return F<LBM_LATTICE_D3Q14, double>::run(c, a...);
        return F<LBM_LATTICE_D3Q14, float>::run(c, a...);
    }
    if (c->precision == PREC_FP64) return F<LBM_LATTICE_D1Q2, double>::run(c, a...);
    return F<LBM_LATTICE_D1Q2, float>::run(c, a...);
}

template <int LAT, typename T> struct StepNd {
    static cudaError_t run(const lbm_nd *c, int src, cudaStream_t s) {
        using C = typename Store<T>::C;
        const unsigned blocks = (unsigned)((c->g.plane + 255) / 256);
        step_nd<LAT, T><<<blocks, 256, 0, s>>>((const T *)c->buf[src], (T *)c->buf[1 - src], c->g,
                                               coef_nd<C>(c));
        return cudaGetLastError();
    }
};
template <int LAT, typename T> struct InitNd {
    static cudaError_t run(const lbm_nd *c, const double *e, const double *q) {
        using C = typename Store<T>::C;
        init_nd<LAT, T><<<grid_of(c->g.plane), 256, 0, c->stream>>>(
            e, q, c->g, c->e_ref, coef_nd<C>(c), (T *)c->buf[1], (T *)c->buf[0]);
        return cudaGetLastError();
    }
};
template <int LAT, typename T> struct MomentsNd {
    static cudaError_t run(const lbm_nd *c, double *e, double *q) {
        using C = typename Store<T>::C;
        moments_nd<LAT, T><<<grid_of(c->g.plane), 256, 0, c->stream>>>(
            (const T *)c->buf[1 - c->cur], c->g, c->n > 0, c->e_ref, 1.0, coef_nd<C>(c), e, q);
        return cudaGetLastError();
    }
};
template <int LAT, typename T> struct PopulationsNd {
    static cudaError_t run(const lbm_nd *c, double *f) {
        const double wa = LAT == LBM_LATTICE_D3Q14 ? 1.0 / 9.0 : 0.5;
        const double wc = LAT == LBM_LATTICE_D3Q14 ? 1.0 / 24.0 : 0.5;
        populations_nd<LAT, T><<<grid_of(c->g.plane), 256, 0, c->stream>>>(
            (const T *)c->buf[1 - c->cur], c->g, c->n > 0, c->e_ref, 1.0, wa, wc, f);
        return cudaGetLastError();
    }
};
template <int LAT, typename T> struct EnergyNd {
    static cudaError_t run(const lbm_nd *c, int) {
        energy_nd<LAT, T><<<ENERGY_BLOCKS, 256, 0, c->stream>>>((const T *)c->buf[1 - c->cur], c->g,
                                                                c->n > 0, c->partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_finalize(c->partials, ENERGY_BLOCKS, c->sums, c->stream);
    }
};

void nd_drop_graphs(lbm_nd *c) {
    for (auto &g : c->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

lbm_status nd_build_graph(lbm_nd *c, int start) {
    NDCK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    int src = start;
    for (int s = 0; s < c->graph_chunk && le == cudaSuccess; ++s) {
        le = nd_dispatch<StepNd>(c, src, c->cap_stream);
        src = 1 - src;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return nd_cuda(c, le, "capture of stream-collide launches");
    }
    if (ee != cudaSuccess) return nd_cuda(c, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&c->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph[start] = nullptr;
        return nd_cuda(c, ie, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

struct NdDevice {
    int old = -1;
    explicit NdDevice(int dev) {
        if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
        else old = -1;
    }
    ~NdDevice() {
        if (old >= 0) cudaSetDevice(old);
    }
};

}  // namespace

extern "C" {

double lbm_nd_lattice_speed(int lattice) {
    if (lattice == LBM_LATTICE_D3Q14) return std::sqrt(3.0 / 5.0);
    if (lattice == LBM_LATTICE_D1Q2) return 1.0 / std::sqrt(3.0);
    return 0.0;
}

lbm_status lbm_nd_create(int lattice, int nx, int ny, int nz, double tau_N, double tau_R,
                         int precision, double e_ref, void *stream, lbm_nd **out) {
    if (!out) return nd_fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (lattice != LBM_LATTICE_D1Q2 && lattice != LBM_LATTICE_D3Q14)
        return nd_fail(nullptr, LBM_EINVAL, "unknown lattice");
    if (nx < 1 || ny < 1 || nz < 1) return nd_fail(nullptr, LBM_EINVAL, "sizes must be >= 1");
    if (lattice == LBM_LATTICE_D1Q2 && (ny != 1 || nz != 1))
        return nd_fail(nullptr, LBM_EINVAL, "a D1Q2 lattice has ny = nz = 1");
    if ((long long)nx * ny * nz > (1LL << 40)) return nd_fail(nullptr, LBM_EINVAL, "too large");
    if (precision == LBM_FP16_DEV || precision == LBM_BF16_DEV)
        return nd_fail(nullptr, LBM_EUNSUPPORTED, "D1Q2 / D3Q14 store FP32 or FP64");
    if (precision != LBM_FP32 && precision != LBM_FP64)
        return nd_fail(nullptr, LBM_EINVAL, "unknown precision");
    if (std::isnan(tau_N) || std::isnan(tau_R) || !(tau_N > 0.0) || !(tau_R > 0.0) ||
        (std::isinf(tau_N) && std::isinf(tau_R)))
        return nd_fail(nullptr, LBM_EINVAL, "tau_N and tau_R must be > 0, not both infinite");
    if (!std::isfinite(e_ref)) return nd_fail(nullptr, LBM_EINVAL, "e_ref is not finite");
    lbm_nd *c = new lbm_nd();
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return nd_fail(nullptr, LBM_ECUDA, "no CUDA device");
    }
    c->lattice = lattice;
    c->dim = lattice == LBM_LATTICE_D3Q14 ? 3 : 1;
    c->Q = lattice == LBM_LATTICE_D3Q14 ? 14 : 2;
    c->precision = precision == LBM_FP64 ? PREC_FP64 : PREC_FP32;
    c->g = Dims{nx, ny, nz, (long long)nx * ny * nz};
    c->tau_N = tau_N;
    c->tau_R = tau_R;
    const double inv_c = (std::isinf(tau_N) ? 0.0 : 1.0 / tau_N) +
                         (std::isinf(tau_R) ? 0.0 : 1.0 / tau_R);
    c->tau = 1.0 / inv_c + 0.5;                                  // Eq. 49
    c->tau_r = tau_R;
    c->kappa = std::isinf(tau_R) ? 1.0 : 2.0 * tau_R / (2.0 * tau_R + 1.0);   // Eq. 54
    c->sigma = std::isinf(tau_R) ? 0.0 : (1.0 - 1.0 / (2.0 * c->tau)) / tau_R;  // Eq. 16
    c->e_ref = e_ref;
    c->stream = (cudaStream_t)stream;
    c->buf_bytes = (size_t)c->Q * (size_t)c->g.plane * (c->precision == PREC_FP64 ? 8 : 4);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&c->buf[i], c->buf_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        lbm_status s = nd_cuda(nullptr, e, "lbm_nd_create");
        lbm_nd_destroy(c);
        return s;
    }
    *out = c;
    return LBM_OK;
}

void lbm_nd_destroy(lbm_nd *c) {
    if (!c) return;
    NdDevice g(c->device);
    if (c->stream || c->buf[0]) cudaStreamSynchronize(c->stream);
    nd_drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaFree(c->buf[0]);
    cudaFree(c->buf[1]);
    cudaFree(c->fields);
    cudaFree(c->partials);
    cudaFree(c->sums);
    delete c;
}

static lbm_status nd_scratch(lbm_nd *c) {
    if (!c->fields)
        NDCK(c, cudaMalloc(&c->fields, sizeof(double) * (1 + c->dim) * (size_t)c->g.plane));
    if (!c->partials) NDCK(c, cudaMalloc(&c->partials, sizeof(double) * 5 * ENERGY_BLOCKS));
    if (!c->sums) NDCK(c, cudaMalloc(&c->sums, sizeof(double) * 5));
    return LBM_OK;
}

lbm_status lbm_nd_init(lbm_nd *c, const double *e, const double *q) {
    NvtxRange nvtx_("lbm_nd_init");
    if (!c) return nd_fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!e) return nd_fail(c, LBM_EINVAL, "e is NULL");
    NdDevice g(c->device);
    if (lbm_status s = nd_scratch(c)) return s;
    const size_t n = (size_t)c->g.plane;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(e[i])) return nd_fail(c, LBM_EINVAL, "e is not finite");
    if (q)
        for (size_t i = 0; i < n * c->dim; ++i)
            if (!std::isfinite(q[i])) return nd_fail(c, LBM_EINVAL, "q is not finite");
    NDCK(c, cudaMemcpyAsync(c->fields, e, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    if (q)
        NDCK(c, cudaMemcpyAsync(c->fields + n, q, sizeof(double) * n * c->dim,
                                cudaMemcpyHostToDevice, c->stream));
    nd_drop_graphs(c);
    NDCK(c, nd_dispatch<InitNd>(c, (const double *)c->fields, q ? (const double *)(c->fields + n)
                                                                : (const double *)nullptr));
    NDCK(c, cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->n = 0;
    c->initialised = true;
    return LBM_OK;
}

lbm_status lbm_nd_step(lbm_nd *c, long n) {
    NvtxRange nvtx_("lbm_nd_step");
    if (!c) return nd_fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (n < 0) return nd_fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->initialised) return nd_fail(c, LBM_EINVAL, "lbm_nd_init has not been called");
    NdDevice g(c->device);
    long left = n;
    if (left >= c->graph_chunk) {
        if (!c->graph[c->cur])
            if (lbm_status s = nd_build_graph(c, c->cur)) return s;
        while (left >= c->graph_chunk) {
            NDCK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
            left -= c->graph_chunk;
            c->n += c->graph_chunk;
        }
    }
    for (; left > 0; --left) {
        NDCK(c, nd_dispatch<StepNd>(c, c->cur, c->stream));
        c->cur = 1 - c->cur;
        c->n += 1;
    }
    return LBM_OK;
}

lbm_status lbm_nd_sync(lbm_nd *c) {
    if (!c) return nd_fail(nullptr, LBM_EINVAL, "ctx is NULL");
    NdDevice g(c->device);
    NDCK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_nd_moments(lbm_nd *c, double *e, double *q) {
    if (!c) return nd_fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return nd_fail(c, LBM_EINVAL, "lbm_nd_init has not been called");
    NdDevice g(c->device);
    if (lbm_status s = nd_scratch(c)) return s;
    const size_t n = (size_t)c->g.plane;
    NDCK(c, nd_dispatch<MomentsNd>(c, c->fields, c->fields + n));
    if (e)
        NDCK(c, cudaMemcpyAsync(e, c->fields, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                c->stream));
    if (q)
        NDCK(c, cudaMemcpyAsync(q, c->fields + n, sizeof(double) * n * c->dim,
                                cudaMemcpyDeviceToHost, c->stream));
    NDCK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_nd_populations(lbm_nd *c, double *f) {
    if (!c) return nd_fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!f) return nd_fail(c, LBM_EINVAL, "f is NULL");
    if (!c->initialised) return nd_fail(c, LBM_EINVAL, "lbm_nd_init has not been called");
    NdDevice g(c->device);
    const size_t bytes = sizeof(double) * (size_t)c->Q * (size_t)c->g.plane;
    double *dev = nullptr;
    NDCK(c, cudaMallocAsync((void **)&dev, bytes, c->stream));
    cudaError_t e = nd_dispatch<PopulationsNd>(c, dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, dev, bytes, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(dev, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return nd_cuda(c, e, "lbm_nd_populations");
    return LBM_OK;
}

lbm_status lbm_nd_energy(lbm_nd *c, double *total) {
    if (!c) return nd_fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return nd_fail(c, LBM_EINVAL, "lbm_nd_init has not been called");
    NdDevice g(c->device);
    if (lbm_status s = nd_scratch(c)) return s;
    NDCK(c, nd_dispatch<EnergyNd>(c, 0));
    double sums[5];
    NDCK(c, cudaMemcpyAsync(sums, c->sums, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
    NDCK(c, cudaStreamSynchronize(c->stream));
    if (total) *total = (double)c->g.plane * c->e_ref + sums[0];
    if (sums[4] > 0.0) return nd_fail(c, LBM_ENONFINITE, "state holds NaN or Inf");
    return LBM_OK;
}

long lbm_nd_step_count(const lbm_nd *c) { return c ? c->n : -1; }

const char *lbm_nd_last_error(const lbm_nd *c) {
    return c ? c->err.c_str() : g_nd_error.c_str();
}

}  // extern "C"
