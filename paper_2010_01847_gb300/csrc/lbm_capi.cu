// C-ABI of the phonon lattice Boltzmann solver (declared in phonon_lbm.h):
// argument checking, device memory, kernel selection, CUDA-graph step
// chunks, read-outs and checkpoints.  All arithmetic of the scheme runs in
// the kernels of stream_collide.cu, staged.cu and readout.cu.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/phonon_lbm.h"
#include "lbm_kernels.h"

using namespace plbm;

struct lbm_ctx {
    int device = 0;
    int nx = 0, ny = 0;
    long long plane = 0;
    int bc_x = 0, bc_y = 0;
    double delta_e = 0.0;
    // sides of LBM_BC_SIDES directions: left, right, bottom, top
    int side_kind[4] = {LBM_SIDE_DIFFUSE, LBM_SIDE_DIFFUSE, LBM_SIDE_DIFFUSE, LBM_SIDE_DIFFUSE};
    double side_val[4] = {0.0, 0.0, 0.0, 0.0};
    double tau_N = 0.0, tau_R = 0.0, tau = 0.0, tau_r = 0.0, kappa = 1.0, sigma = 0.0;
    int precision = 0;
    int rounding = LBM_ROUND_NEAREST;   // 16-bit storage only
    double e_ref = 1.0;
    double scale = 1.0;
    cudaStream_t stream = nullptr;
    void *buf[2] = {nullptr, nullptr};
    bool owns_buf = false;
    size_t buf_bytes = 0;
    int cur = 0;           // buffer with the post-collision populations of step n
    long n = 0;            // steps since lbm_init
    bool initialised = false;
    int kernel = KERNEL_SCALAR;
    StagedPlan plan;            // launch shape of the staged kernel
    int stages_req = 0, ctas_req = 0, cw_req = 0, hint_req = 0;
    ResidentPlan rplan;         // launch shape of the cluster-resident kernel
    int cluster_req = 0;
    int wave_steps = 4;         // multi-step kernel: steps per launch
    int wave_rows = 128;        // and rows per strip segment
    int graph_chunk = 64;
    // launch timing (lbm_set_launch_timing): event pairs around launches
    bool timing = false;
    struct Timed { cudaEvent_t a, b; int which; long steps; };
    std::vector<Timed> timed;
    double timed_ms[3] = {0.0, 0.0, 0.0};
    long long timed_launches[3] = {0, 0, 0}, timed_steps[3] = {0, 0, 0};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    void *prev = nullptr;       // residual history, 3 planes of the compute type
    bool have_prev = false;
    long prev_step = 0;
    double *fields = nullptr;   // 3 planes of doubles: init staging / read-outs
    double *partials = nullptr; // 5 doubles per block of the widest reduction launch
    long long partial_blocks = 0;
    double *aux = nullptr;      // [0..4] sums, [5] max-deviation bits, [6] status word
    long long launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

constexpr uint64_t STATE_MAGIC = 0x314d424c4e4f4850ULL;   // "PHONLBM1"

struct StateHeader {
    uint64_t magic;
    int32_t version, nx, ny, precision, bc_x, bc_y, cur, pad;
    int64_t n;
    double scale;
    uint64_t buf_bytes;
};

size_t elem_size(int precision) {
    switch (precision) {
        case PREC_FP32: return 4;
        case PREC_FP64: return 8;
        default: return 2;
    }
}

lbm_status fail(lbm_ctx *ctx, lbm_status s, const std::string &msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_error = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx *ctx, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                      cudaGetErrorString(e) + ")";
    // the error is reported here; clear the runtime's per-thread record of it
    // so a later call does not pick it up again (sticky errors persist anyway)
    (void)cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(ctx, LBM_ENOMEM, msg);
    return fail(ctx, LBM_ECUDA, msg);
}

#define CK(ctx, call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
        else old = -1;
    }
    ~DeviceGuard() {
        if (old >= 0) cudaSetDevice(old);
    }
};

template <typename C>
Coef<C> make_coef(const lbm_ctx *c) {
    // Eqs. 13, 15-18, 54 and 58 as the coefficients of lbm_device.cuh.
    Coef<C> k{};
    k.omega = (C)(1.0 / c->tau);
    k.sigma = (C)c->sigma;
    const double lambda = std::isinf(c->tau_r) ? 0.0 : 1.0 / (2.0 * c->tau_r + 1.0);
    k.lambda = (C)lambda;
    k.zeta = (C)(lambda + c->sigma * c->tau * (1.0 - lambda));
    k.w_axis = (C)(2.0 / 9.0);
    k.w_diag = (C)0.25 - k.w_axis;                  // exact: 4 w_axis + 4 w_diag = 1
    k.h_axis = (C)(1.0 / 3.0);
    k.h_diag = ((C)1 - (C)2 * k.h_axis) / (C)4;     // exact: 2 h_axis + 4 h_diag = 1
    k.u_axis = (C)0.8;
    k.u_diag = ((C)1 - k.u_axis) / (C)2;            // exact: u_axis + 2 u_diag = 1
    k.jump_axis = (C)(c->scale * (2.0 / 9.0) * c->delta_e);
    k.jump_diag = (C)(c->scale * (1.0 / 36.0) * c->delta_e);
    // Eq. 55 on deviations: s w_i (e_s - e_ref); Eq. 57: s q_0 / kappa
    for (int sd = 0; sd < 4; ++sd) {
        const int kind = c->side_kind[sd];
        const double v = c->side_val[sd];
        k.side_kind[sd] = kind;
        k.side_axis[sd] = (C)(kind == LBM_SIDE_ISOTHERMAL ? c->scale * (2.0 / 9.0) * (v - c->e_ref)
                                                          : 0.0);
        k.side_diag[sd] = (C)(kind == LBM_SIDE_ISOTHERMAL ? c->scale * (1.0 / 36.0) * (v - c->e_ref)
                                                          : 0.0);
        k.side_flux[sd] = (C)(kind == LBM_SIDE_HEAT_FLUX ? c->scale * v / c->kappa : 0.0);
    }
    set_tile_refs(k, c->precision, c->nx, c->ny, c->tau, c->tau_r);
    k.stochastic = c->rounding == LBM_ROUND_STOCHASTIC ? 1 : 0;
    return k;
}

bool has_sides(const lbm_ctx *c) { return c->bc_x == LBM_BC_SIDES || c->bc_y == LBM_BC_SIDES; }

// Largest |d_i| / s a side can write: w_axis |e_s - e_ref| for an isothermal
// side, about |q_0| / kappa for a heat-flux side.
double side_bound(const lbm_ctx *c, int kind, double v) {
    if (kind == LBM_SIDE_ISOTHERMAL) return (2.0 / 9.0) * std::fabs(v - c->e_ref);
    if (kind == LBM_SIDE_HEAT_FLUX) return std::fabs(v) / c->kappa;
    return 0.0;
}

// A corner node between a BC_SIDES x side and a y side (walls or a side)
// receives unknown populations from both directions; the scheme fixes them
// only when one of its sides is isothermal (Eq. 55 sets the whole node).
lbm_status check_corners(lbm_ctx *c) {
    if (c->bc_x != LBM_BC_SIDES ||
        (c->bc_y != LBM_BC_SIDES && c->bc_y != LBM_BC_DIFFUSE_WALLS))
        return LBM_OK;
    static const char *xname[2] = {"left", "right"}, *yname[2] = {"bottom", "top"};
    for (int xs = 0; xs < 2; ++xs)
        for (int ys = 0; ys < 2; ++ys) {
            const bool iso = c->side_kind[xs] == LBM_SIDE_ISOTHERMAL ||
                             (c->bc_y == LBM_BC_SIDES && c->side_kind[2 + ys] == LBM_SIDE_ISOTHERMAL);
            if (!iso)
                return fail(c, LBM_EUNSUPPORTED,
                            std::string("the ") + xname[xs] + "-" + yname[ys] +
                                " corner touches no isothermal side; the scheme defines no "
                                "treatment for it");
        }
    return LBM_OK;
}

Readout make_readout(const lbm_ctx *c) {
    Readout r;
    r.nx = c->nx;
    r.ny = c->ny;
    r.bc_x = c->bc_x;
    r.bc_y = c->bc_y;
    r.pulled = c->n > 0;
    r.e_ref = c->e_ref;
    r.inv_scale = 1.0 / c->scale;
    r.kappa = c->kappa;
    return r;
}

// Calls F<T>(ctx...) for the context's storage type.
template <template <typename> class F, typename... A>
cudaError_t dispatch(const lbm_ctx *c, A... a) {
    switch (c->precision) {
        case PREC_FP32: return F<float>::run(c, a...);
        case PREC_FP64: return F<double>::run(c, a...);
        case PREC_FP16: return F<__half>::run(c, a...);
        default: return F<__nv_bfloat16>::run(c, a...);
    }
}

int *status_word(const lbm_ctx *c) { return (int *)(c->aux + 6); }
// the middle level of the two-pass residual total, after the block partials
double *mid_ptr(const lbm_ctx *c) { return c->partials + 5 * c->partial_blocks; }
double *sums_ptr(const lbm_ctx *c) { return c->aux; }

template <typename T> struct StepOp {
    static cudaError_t run(const lbm_ctx *c, int src, cudaStream_t s) {
        using C = typename Store<T>::C;
        if constexpr (std::is_same<T, float>::value)
            if (c->kernel == KERNEL_RESIDENT)     // one step: last -> dst, previous -> src
                return launch_resident((const float *)c->buf[src], (float *)c->buf[1 - src],
                                       (float *)c->buf[src], c->nx, c->ny, c->bc_x, c->bc_y,
                                       make_coef<float>(c), 1, c->rplan, status_word(c), s);
        return launch_step<T>(c->kernel, (const T *)c->buf[src], (T *)c->buf[1 - src], c->nx,
                              c->ny, c->bc_x, c->bc_y, make_coef<C>(c), status_word(c), nullptr,
                              c->plan, nullptr, s);
    }
};
// One step that also reduces the residual sums of the state it pulls.
template <typename T> struct StepResidualOp {
    static cudaError_t run(const lbm_ctx *c, int src, int *blocks) {
        using C = typename Store<T>::C;
        ResidualReq<C> rq;
        rq.prev = (C *)c->prev;
        rq.have_prev = c->have_prev ? 1 : 0;
        rq.inv_scale = (C)(1.0 / c->scale);
        rq.partials = c->partials;
        return launch_step<T>(c->kernel, (const T *)c->buf[src], (T *)c->buf[1 - src], c->nx,
                              c->ny, c->bc_x, c->bc_y, make_coef<C>(c), status_word(c), &rq,
                              c->plan, blocks, c->stream);
    }
};
template <typename T> struct MomentsOp {
    static cudaError_t run(const lbm_ctx *c, double *e, double *qx, double *qy) {
        using C = typename Store<T>::C;
        return launch_moments<T>((const T *)c->buf[1 - c->cur], make_readout(c), make_coef<C>(c),
                                 e, qx, qy, c->stream);
    }
};
template <typename T> struct PopulationsOp {
    static cudaError_t run(const lbm_ctx *c, double *f) {
        using C = typename Store<T>::C;
        return launch_populations<T>((const T *)c->buf[1 - c->cur], make_readout(c),
                                     make_coef<C>(c), f, c->stream);
    }
};
template <typename T> struct ResidualOp {
    static cudaError_t run(const lbm_ctx *c, int dummy) {
        (void)dummy;
        using C = typename Store<T>::C;
        return launch_residual<T>((const T *)c->buf[1 - c->cur], make_readout(c),
                                  make_coef<C>(c), (C *)c->prev, c->have_prev, c->partials,
                                  sums_ptr(c), c->stream, mid_ptr(c));
    }
};
template <typename T> struct InitOp {
    static cudaError_t run(const lbm_ctx *c, const double *e, const double *qx,
                           const double *qy) {
        using C = typename Store<T>::C;
        // step 0 state -> buffer 1, its collision -> buffer 0 (cur = 0)
        return launch_init<T>(e, qx, qy, c->nx, c->ny, c->e_ref, c->scale, make_coef<C>(c),
                              (T *)c->buf[1], (T *)c->buf[0], c->stream);
    }
};

void drop_graphs(lbm_ctx *c) {
    for (int i = 0; i < 2; ++i) {
        if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
        c->graph[i] = nullptr;
    }
}

size_t compute_size(int precision) { return precision == PREC_FP64 ? 8 : 4; }

lbm_status ensure_scratch(lbm_ctx *c, bool need_prev) {
    if (!c->fields) CK(c, cudaMalloc(&c->fields, sizeof(double) * 3 * (size_t)c->plane));
    if (!c->aux) {
        CK(c, cudaMalloc(&c->aux, sizeof(double) * 8));
        CK(c, cudaMemset(c->aux, 0, sizeof(double) * 8));
    }
    if (need_prev) {
        long long blocks = step_blocks(c->kernel, c->precision, c->nx, c->ny, c->plan);
        const long long rb = readout_blocks(c->precision, c->nx, c->ny, c->bc_x, c->bc_y);
        if (blocks < rb) blocks = rb;
        if (blocks > c->partial_blocks) {
            cudaFree(c->partials);
            c->partials = nullptr;
            c->partial_blocks = 0;
            // + FINALIZE_MID records: the middle level of the two-pass total
            CK(c, cudaMalloc(&c->partials, sizeof(double) * 5 * (size_t)(blocks + FINALIZE_MID)));
            c->partial_blocks = blocks;
        }
        if (!c->prev)
            CK(c, cudaMalloc(&c->prev, compute_size(c->precision) * 3 * (size_t)c->plane));
    }
    return LBM_OK;
}

// Reads the device status word (after the stream is synchronised).
lbm_status check_status(lbm_ctx *c) {
    if (!c->aux) return LBM_OK;
    int st = 0;
    CK(c, cudaMemcpy(&st, status_word(c), sizeof(int), cudaMemcpyDeviceToHost));
    if (st)
        return fail(c, LBM_ETIMEOUT,
                    (st & 2) ? "a bounded device-side wait gave up (cluster-resident kernel)"
                             : "a bounded device-side wait gave up (staged kernel)");
    return LBM_OK;
}

// Residual and energy from the 5 device sums (same formulas for the
// stand-alone and the fused pass).
lbm_status finish_residual(lbm_ctx *c, const double (&sums)[5], double *r,
                           double *total_energy) {
    const double n = (double)c->plane;
    const double mean = sums[0] / n;
    const double var_e = std::fmax(sums[1] - n * mean * mean, 0.0);
    const double denom = std::sqrt(var_e + sums[2]);
    const long k = c->n - c->prev_step;
    double res = INFINITY;
    if (c->have_prev && k > 0) {
        const double num = std::sqrt(sums[3]);
        res = denom > 0.0 ? num / ((double)k * denom) : (num == 0.0 ? 0.0 : INFINITY);
    }
    c->have_prev = true;
    c->prev_step = c->n;
    if (r) *r = res;
    if (total_energy) *total_energy = n * c->e_ref + sums[0];
    if (sums[4] > 0.0) return fail(c, LBM_ENONFINITE, "state holds NaN or Inf");
    return LBM_OK;
}

constexpr long long RESIDENT_AUTO_NODES = 16384;
constexpr long long WAVE_AUTO_NODES = 1LL << 24;

// Works out the cluster-resident plan (FP32 lattices whose two buffers fit
// in one cluster's shared memory); false when there is none.
bool resident_ok(lbm_ctx *c) {
    ResidentPlan p;
    if (resident_plan(c->precision, c->nx, c->ny, c->cluster_req, &p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    c->rplan = p;
    return true;
}

int resolve_kernel(lbm_ctx *c, int requested) {
    const bool vec_ok = c->nx % vector_width(c->precision) == 0;
    // plain 16-bit steps on the vector layout run the pipelined kernel, set
    // up here, outside any stream capture
    if (vec_ok && has_tile_refs(c->precision) && prepare_pipe16(c->precision) != cudaSuccess)
        (void)cudaGetLastError();
    // without timing: small FP32 lattices run cluster-resident, n steps per
    // launch (measured 1.5-2.4x faster than one launch per step up to 16384
    // nodes; beyond that 16 SMs do less than the whole GPU)
    if (requested == KERNEL_AUTO && c->precision == PREC_FP32 &&
        c->plane <= RESIDENT_AUTO_NODES && resident_ok(c))
        return KERNEL_RESIDENT;
    // small FP64 lattices: FP64 arithmetic bounds the step, and one node per
    // thread spreads it over twice the SMs of the 2-node vectors (128 x 32:
    // 5.3-5.6 against 6.2 us per step)
    if (requested == KERNEL_AUTO && c->precision == PREC_FP64 && c->plane <= RESIDENT_AUTO_NODES)
        return KERNEL_SCALAR;
    if (requested == KERNEL_WAVE) {
        if (!wave_supported(c->precision, c->nx, c->ny, c->bc_x, c->bc_y)) return -1;
        if (c->wave_steps > wave_max_steps(c->precision))
            c->wave_steps = wave_max_steps(c->precision);
        return KERNEL_WAVE;
    }
    if (has_sides(c)) {     // the per-side rules: scalar, vector and resident kernels
        if (requested == KERNEL_AUTO) return vec_ok ? KERNEL_VECTOR : KERNEL_SCALAR;
        if (requested == KERNEL_SCALAR) return KERNEL_SCALAR;
        if (requested == KERNEL_RESIDENT) return resident_ok(c) ? KERNEL_RESIDENT : -1;
        return (requested == KERNEL_VECTOR && vec_ok) ? KERNEL_VECTOR : -1;
    }
    // the staged kernel also needs its plan (launch attributes, occupancy)
    // worked out on this device, here, outside any stream capture
    const int cw = c->cw_req > 0 ? c->cw_req : 8;
    bool staged_ok = staged_supported(c->precision, c->nx, c->ny, cw);
    if (staged_ok) {
        StagedPlan p;
        staged_ok = staged_plan(c->precision, c->stages_req, c->ctas_req, cw, c->hint_req, &p) ==
                    cudaSuccess;
        if (staged_ok) c->plan = p;
        else (void)cudaGetLastError();
    }
    if (requested == KERNEL_AUTO) {
        // without timing (lbm_autotune times them): large lattices the
        // multi-step kernel where it applies (FP32: 5 steps per launch,
        // 128-row segments, 424 against 105 GLUPS at 8192^2; 16-bit: 4
        // steps, 256-row segments, 340 against 171; from 16 M nodes its
        // strip-segments fill the GPU), else
        // the vector kernel, the fastest single-step
        // kernel measured at 8192^2 for every storage kind (FP32 6.7, 16-bit
        // 6.5 TB/s against the staged kernel's 5.7 and 6.0), with the least
        // set-up for small, launch-latency bound lattices
        if (c->plane >= WAVE_AUTO_NODES && c->nx >= 256 &&
            wave_supported(c->precision, c->nx, c->ny, c->bc_x, c->bc_y)) {
            const bool fp32 = c->precision == PREC_FP32;
            c->wave_steps = fp32 ? 5 : 4;
            c->wave_rows = fp32 ? 128 : 256;
            return KERNEL_WAVE;
        }
        return vec_ok ? KERNEL_VECTOR : KERNEL_SCALAR;
    }
    if (requested == KERNEL_VECTOR && !vec_ok) return -1;
    if (requested == KERNEL_STAGED && !staged_ok) return -1;
    if (requested == KERNEL_RESIDENT && !resident_ok(c)) return -1;
    return requested;
}

lbm_status create_common(lbm_grid g, double tau_N, double tau_R, lbm_boundary bc,
                         lbm_precision precision, double e_ref, void *stream, void *buf_a,
                         void *buf_b, size_t buf_bytes, lbm_ctx **out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (g.nx < 1 || g.ny < 1) return fail(nullptr, LBM_EINVAL, "grid must be at least 1x1");
    if ((long long)g.nx * g.ny > (1LL << 40))
        return fail(nullptr, LBM_EINVAL, "grid too large");
    if (bc.x == LBM_BC_DIFFUSE_WALLS)
        return fail(nullptr, LBM_EUNSUPPORTED, "diffuse walls are supported on y only");
    if (bc.y == LBM_BC_PERIODIC_GRADIENT)
        return fail(nullptr, LBM_EUNSUPPORTED,
                    "the periodic temperature gradient is supported on x only");
    if ((bc.x != LBM_BC_PERIODIC && bc.x != LBM_BC_PERIODIC_GRADIENT && bc.x != LBM_BC_SIDES) ||
        (bc.y != LBM_BC_PERIODIC && bc.y != LBM_BC_DIFFUSE_WALLS && bc.y != LBM_BC_SIDES))
        return fail(nullptr, LBM_EINVAL, "unknown boundary kind");
    if (bc.y == LBM_BC_DIFFUSE_WALLS && g.ny < 2)
        return fail(nullptr, LBM_EINVAL, "diffuse walls need ny >= 2");
    if ((bc.x == LBM_BC_SIDES && g.nx < 2) || (bc.y == LBM_BC_SIDES && g.ny < 2))
        return fail(nullptr, LBM_EINVAL, "a direction with two sides needs at least 2 nodes");
    if (!std::isfinite(bc.delta_e)) return fail(nullptr, LBM_EINVAL, "delta_e is not finite");
    if (!std::isfinite(e_ref)) return fail(nullptr, LBM_EINVAL, "e_ref is not finite");
    if (std::isnan(tau_N) || std::isnan(tau_R) || !(tau_N > 0.0) || !(tau_R > 0.0))
        return fail(nullptr, LBM_EINVAL, "tau_N and tau_R must be > 0");
    if (std::isinf(tau_N) && std::isinf(tau_R))
        return fail(nullptr, LBM_EINVAL, "tau_N and tau_R cannot both be infinite");
    if (precision < LBM_FP32 || precision > LBM_FP64)
        return fail(nullptr, LBM_EINVAL, "unknown precision");

    lbm_ctx *c = new lbm_ctx();
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    c->nx = g.nx;
    c->ny = g.ny;
    c->plane = (long long)g.nx * g.ny;
    c->bc_x = bc.x;
    c->bc_y = bc.y;
    c->delta_e = bc.delta_e;
    c->tau_N = tau_N;
    c->tau_R = tau_R;
    // Section 2.1: 1/tau_C = 1/tau_N + 1/tau_R; Eq. 49: tau = tau_C + 1/2;
    // Section 2.4: tau_r = tau_R; Eq. 54: kappa; Eq. 16: sigma.
    const double inv_c = (std::isinf(tau_N) ? 0.0 : 1.0 / tau_N) +
                         (std::isinf(tau_R) ? 0.0 : 1.0 / tau_R);
    c->tau = 1.0 / inv_c + 0.5;
    c->tau_r = tau_R;
    c->kappa = std::isinf(tau_R) ? 1.0 : 2.0 * tau_R / (2.0 * tau_R + 1.0);
    c->sigma = std::isinf(tau_R) ? 0.0 : (1.0 - 1.0 / (2.0 * c->tau)) / tau_R;
    c->precision = precision;
    c->e_ref = e_ref;
    c->stream = (cudaStream_t)stream;
    c->buf_bytes = lbm_population_bytes(g, precision);

    if (buf_a || buf_b) {
        if (!buf_a || !buf_b || buf_a == buf_b) {
            delete c;
            return fail(nullptr, LBM_EINVAL, "need two distinct caller buffers");
        }
        if (buf_bytes < c->buf_bytes) {
            delete c;
            return fail(nullptr, LBM_EINVAL, "caller buffers are too small");
        }
        if (((uintptr_t)buf_a | (uintptr_t)buf_b) & 255u) {
            delete c;
            return fail(nullptr, LBM_EINVAL, "caller buffers must be 256-byte aligned");
        }
        c->buf[0] = buf_a;
        c->buf[1] = buf_b;
        c->owns_buf = false;
    } else {
        for (int i = 0; i < 2; ++i) {
            e = cudaMalloc(&c->buf[i], c->buf_bytes);
            if (e != cudaSuccess) {
                lbm_status s = cuda_fail(nullptr, e, "cudaMalloc(population buffer)");
                if (c->buf[0]) cudaFree(c->buf[0]);
                delete c;
                return s;
            }
        }
        c->owns_buf = true;
    }
    e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        lbm_status s = cuda_fail(nullptr, e, "cudaStreamCreateWithFlags");
        lbm_destroy(c);
        return s;
    }
    c->kernel = resolve_kernel(c, KERNEL_AUTO);
    *out = c;
    return LBM_OK;
}

lbm_status init_from_device(lbm_ctx *c, const double *e, const double *qx, const double *qy) {
    if (lbm_status s = ensure_scratch(c, false)) return s;
    unsigned long long *maxbits = (unsigned long long *)(c->aux + 5);
    CK(c, cudaMemsetAsync(c->aux, 0, sizeof(double) * 8, c->stream));   // also clears status
    CK(c, launch_max_deviation(e, qx, qy, c->plane, c->e_ref, maxbits, c->stream));
    unsigned long long bits = 0;
    CK(c, cudaMemcpyAsync(&bits, maxbits, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    double amax;
    std::memcpy(&amax, &bits, sizeof(amax));
    if (!std::isfinite(amax)) return fail(c, LBM_EINVAL, "initial fields are not finite");
    c->scale = 1.0;
    if (c->precision == PREC_FP16 || c->precision == PREC_BF16) {
        // largest |d_i| ~ 2^12 after scaling: room for 16x growth below the
        // FP16 maximum, far above its smallest normal number
        double a = std::fmax(amax, (2.0 / 9.0) * std::fabs(c->delta_e));
        if (has_sides(c))
            for (int sd = 0; sd < 4; ++sd)
                a = std::fmax(a, side_bound(c, c->side_kind[sd], c->side_val[sd]));
        if (a > 0.0) {
            int ex;
            std::frexp(a, &ex);        // a < 2^ex
            int p = 12 - ex;
            p = p > 100 ? 100 : (p < -100 ? -100 : p);
            c->scale = std::ldexp(1.0, p);
        }
    }
    drop_graphs(c);
    CK(c, dispatch<InitOp>(c, e, qx, qy));
    c->cur = 0;
    c->n = 0;
    c->have_prev = false;
    c->prev_step = 0;
    c->launches = 0;
    c->initialised = true;
    return LBM_OK;
}

// One multi-step launch of `steps` steps from buffer src.
cudaError_t wave_launch(const lbm_ctx *c, int src, int steps, cudaStream_t s) {
    if (c->precision == PREC_FP32)
        return launch_step_wave(steps, (const float *)c->buf[src], (float *)c->buf[1 - src],
                                c->nx, c->ny, c->bc_x, c->bc_y, make_coef<float>(c),
                                c->wave_rows, s);
    return launch_step_wave16(c->precision, steps, c->buf[src], c->buf[1 - src], c->nx, c->ny,
                              c->bc_x, c->bc_y, make_coef<float>(c), c->wave_rows, s);
}

// Launches in one captured graph of multi-step launches: an even number (the
// buffers end where they began) of about graph_chunk steps.
int wave_graph_launches(const lbm_ctx *c) {
    const int pairs = c->graph_chunk / (2 * c->wave_steps);
    return 2 * (pairs > 1 ? pairs : 1);
}

lbm_status build_graph(lbm_ctx *c, int start) {
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int src = start;
    cudaError_t le = cudaSuccess;
    if (c->kernel == KERNEL_WAVE) {
        for (int s = 0; s < wave_graph_launches(c) && le == cudaSuccess; ++s) {
            le = wave_launch(c, src, c->wave_steps, c->cap_stream);
            src = 1 - src;
        }
    } else {
        for (int s = 0; s < c->graph_chunk && le == cudaSuccess; ++s) {
            le = dispatch<StepOp>(c, src, c->cap_stream);
            src = 1 - src;
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, le, "capture of stream-collide launches");
    }
    if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&c->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph[start] = nullptr;
        return cuda_fail(c, ie, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

// Launch timing: which = 0 multi-step launches, 1 single steps, 2 steps
// that also reduce the residual.  timed_begin records the opening event of
// a launch (or returns a null record when timing is off), timed_end the
// closing one.
enum { TIMED_WAVE = 0, TIMED_SINGLE = 1, TIMED_RESIDUAL = 2 };

cudaError_t timed_begin(lbm_ctx *c, int which, long steps, int *slot) {
    *slot = -1;
    if (!c->timing) return cudaSuccess;
    lbm_ctx::Timed t{nullptr, nullptr, which, steps};
    cudaError_t e = cudaEventCreate(&t.a);
    if (e == cudaSuccess) e = cudaEventCreate(&t.b);
    if (e == cudaSuccess) e = cudaEventRecord(t.a, c->stream);
    if (e != cudaSuccess) {
        if (t.a) cudaEventDestroy(t.a);
        if (t.b) cudaEventDestroy(t.b);
        return e;
    }
    c->timed.push_back(t);
    *slot = (int)c->timed.size() - 1;
    return cudaSuccess;
}

cudaError_t timed_end(lbm_ctx *c, int slot) {
    if (slot < 0) return cudaSuccess;
    return cudaEventRecord(c->timed[slot].b, c->stream);
}

// Folds the recorded launches into the totals (after the stream is
// synchronised) and releases their events.
cudaError_t timed_collect(lbm_ctx *c) {
    cudaError_t err = cudaSuccess;
    for (auto &t : c->timed) {
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t.a, t.b);
        if (err == cudaSuccess) {
            c->timed_ms[t.which] += ms;
            c->timed_launches[t.which] += 1;
            c->timed_steps[t.which] += t.steps;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->timed.clear();
    return err;
}

lbm_status single_step(lbm_ctx *c) {
    int slot;
    CK(c, timed_begin(c, TIMED_SINGLE, 1, &slot));
    CK(c, dispatch<StepOp>(c, c->cur, c->stream));
    CK(c, timed_end(c, slot));
    c->cur = 1 - c->cur;
    c->n += 1;
    c->launches += 1;
    return LBM_OK;
}

// Advances n steps.  With the multi-step kernel a launch of k steps leaves
// the post-collision state of its last step only; the read-outs need the one
// of the step before too (they pull it), so a call that ends readable
// (end_readable) finishes with a single step, and lbm_step_residual's plain
// steps end without one, as its own last step is a single step.
lbm_status advance(lbm_ctx *c, long n, bool end_readable) {
    if (n <= 0) return LBM_OK;
    if (c->kernel == KERNEL_RESIDENT) {
        // all n steps in one launch; the buffers end as n single steps leave them
        const int last = c->cur ^ (int)(n & 1);
        CK(c, launch_resident((const float *)c->buf[c->cur], (float *)c->buf[last],
                              (float *)c->buf[last ^ 1], c->nx, c->ny, c->bc_x, c->bc_y,
                              make_coef<float>(c), n, c->rplan, status_word(c), c->stream));
        c->cur = last;
        c->n += n;
        c->launches += 1;
        return LBM_OK;
    }
    if (c->kernel == KERNEL_WAVE) {
        const long tail = end_readable ? 1 : 0;
        long m = n - tail;
        const int K = c->wave_steps;
        const int gl = wave_graph_launches(c);
        if (!c->timing && c->graph_chunk > 0 && m >= (long)gl * K) {
            if (!c->graph[c->cur])
                if (lbm_status s = build_graph(c, c->cur)) return s;
            while (m >= (long)gl * K) {      // an even number of launches: cur unchanged
                CK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
                m -= (long)gl * K;
                c->n += (long)gl * K;
                c->launches += gl;
            }
        }
        while (m >= WAVE_MIN_STEPS) {
            const int k = m >= K ? K : (int)m;
            int slot;
            CK(c, timed_begin(c, TIMED_WAVE, k, &slot));
            CK(c, wave_launch(c, c->cur, k, c->stream));
            CK(c, timed_end(c, slot));
            c->cur = 1 - c->cur;
            m -= k;
            c->n += k;
            c->launches += 1;
        }
        for (long i = 0; i < m + tail; ++i)
            if (lbm_status s = single_step(c)) return s;
        return LBM_OK;
    }
    long left = n;
    if (!c->timing && c->graph_chunk > 0 && left >= c->graph_chunk) {
        if (!c->graph[c->cur])
            if (lbm_status s = build_graph(c, c->cur)) return s;
        while (left >= c->graph_chunk) {
            CK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
            left -= c->graph_chunk;
            c->n += c->graph_chunk;
            c->launches += c->graph_chunk;
        }
    }
    for (; left > 0; --left)
        if (lbm_status s = single_step(c)) return s;
    return LBM_OK;
}

}  // namespace

void plbm::set_global_error(const char *msg) { g_create_error = msg; }

extern "C" {

double lbm_tau_from_kn(double kn, double length) { return kn * length * std::sqrt(3.0 / 5.0); }

size_t lbm_population_bytes(lbm_grid grid, lbm_precision precision) {
    if (grid.nx < 1 || grid.ny < 1 || precision < LBM_FP32 || precision > LBM_FP64) return 0;
    return (size_t)state_elems(precision, grid.nx, grid.ny) * elem_size(precision);
}

lbm_status lbm_create(lbm_grid grid, double tau_N, double tau_R, lbm_boundary bc,
                      lbm_precision precision, double e_ref, void *stream, lbm_ctx **out) {
    return create_common(grid, tau_N, tau_R, bc, precision, e_ref, stream, nullptr, nullptr, 0,
                         out);
}

lbm_status lbm_create_ex(lbm_grid grid, double tau_N, double tau_R, lbm_boundary bc,
                         lbm_precision precision, double e_ref, void *stream, void *buf_a,
                         void *buf_b, size_t buf_bytes, lbm_ctx **out) {
    if (!buf_a || !buf_b) return fail(nullptr, LBM_EINVAL, "caller buffers are NULL");
    return create_common(grid, tau_N, tau_R, bc, precision, e_ref, stream, buf_a, buf_b,
                         buf_bytes, out);
}

void lbm_destroy(lbm_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (auto &t : c->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->owns_buf) {
        cudaFree(c->buf[0]);
        cudaFree(c->buf[1]);
    }
    cudaFree(c->prev);
    cudaFree(c->fields);
    cudaFree(c->partials);
    cudaFree(c->aux);
    delete c;
}

lbm_status lbm_init(lbm_ctx *c, const double *e, const double *qx, const double *qy) {
    NvtxRange nvtx_("lbm_init");
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!e) return fail(c, LBM_EINVAL, "e is NULL");
    DeviceGuard g(c->device);
    const long long n = c->plane;
    const double *src[3] = {e, qx, qy};
    // non-finite inputs are caught on the device by the scale pass
    if (lbm_status s = ensure_scratch(c, false)) return s;
    for (int f = 0; f < 3; ++f)
        if (src[f])
            CK(c, cudaMemcpyAsync(c->fields + f * n, src[f], sizeof(double) * n,
                                  cudaMemcpyHostToDevice, c->stream));
    return init_from_device(c, c->fields, qx ? c->fields + n : nullptr,
                            qy ? c->fields + 2 * n : nullptr);
}

lbm_status lbm_init_device(lbm_ctx *c, const double *e, const double *qx, const double *qy) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!e) return fail(c, LBM_EINVAL, "e is NULL");
    DeviceGuard g(c->device);
    return init_from_device(c, e, qx, qy);
}

lbm_status lbm_step(lbm_ctx *c, long n) {
    NvtxRange nvtx_("lbm_step");
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    if (lbm_status s = check_corners(c)) return s;
    DeviceGuard g(c->device);
    return advance(c, n, true);
}

lbm_status lbm_sync(lbm_ctx *c) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    DeviceGuard g(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaGetLastError());
    return check_status(c);
}

lbm_status lbm_moments_device(lbm_ctx *c, double *e, double *qx, double *qy) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    if (c->n > 0)
        if (lbm_status s = check_corners(c)) return s;
    DeviceGuard g(c->device);
    if (!e && !qx && !qy) return LBM_OK;
    CK(c, dispatch<MomentsOp>(c, e, qx, qy));
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *c, double *e, double *qx, double *qy) {
    NvtxRange nvtx_("lbm_moments");
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    if (c->n > 0)
        if (lbm_status s = check_corners(c)) return s;
    DeviceGuard g(c->device);
    if (!e && !qx && !qy) return LBM_OK;
    if (lbm_status s = ensure_scratch(c, false)) return s;
    const long long n = c->plane;
    double *d[3] = {c->fields, c->fields + n, c->fields + 2 * n};
    CK(c, dispatch<MomentsOp>(c, d[0], d[1], d[2]));
    double *h[3] = {e, qx, qy};
    for (int f = 0; f < 3; ++f)
        if (h[f])
            CK(c, cudaMemcpyAsync(h[f], d[f], sizeof(double) * n, cudaMemcpyDeviceToHost,
                                  c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_populations(lbm_ctx *c, double *f) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    if (c->n > 0)
        if (lbm_status s = check_corners(c)) return s;
    DeviceGuard g(c->device);
    double *dev = nullptr;
    CK(c, cudaMallocAsync((void **)&dev, sizeof(double) * 8 * (size_t)c->plane, c->stream));
    cudaError_t e = dispatch<PopulationsOp>(c, dev);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, dev, sizeof(double) * 8 * (size_t)c->plane,
                            cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(dev, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_populations");
    return LBM_OK;
}

lbm_status lbm_residual(lbm_ctx *c, double *r, double *total_energy) {
    NvtxRange nvtx_("lbm_residual");
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    if (c->n > 0)
        if (lbm_status s = check_corners(c)) return s;
    DeviceGuard g(c->device);
    if (lbm_status s = ensure_scratch(c, true)) return s;
    CK(c, dispatch<ResidualOp>(c, 0));
    double sums[5];
    CK(c, cudaMemcpyAsync(sums, sums_ptr(c), sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (lbm_status s = check_status(c)) return s;
    return finish_residual(c, sums, r, total_energy);
}

lbm_status lbm_step_residual(lbm_ctx *c, long n, double *r, double *total_energy) {
    NvtxRange nvtx_("lbm_step_residual");
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    if (c->n > 0)
        if (lbm_status s = check_corners(c)) return s;
    if (n == 0) return lbm_residual(c, r, total_energy);
    DeviceGuard g(c->device);
    if (lbm_status s = ensure_scratch(c, true)) return s;
    if (lbm_status s = check_corners(c)) return s;
    if (lbm_status s = advance(c, n - 1, false)) return s;
    int blocks = 0;
    int slot;
    CK(c, timed_begin(c, TIMED_RESIDUAL, 1, &slot));
    CK(c, dispatch<StepResidualOp>(c, c->cur, &blocks));
    CK(c, timed_end(c, slot));
    c->cur = 1 - c->cur;
    c->n += 1;
    c->launches += 1;
    int fin = 0;
    CK(c, launch_finalize(c->partials, blocks, sums_ptr(c), c->stream, mid_ptr(c), &fin));
    c->launches += fin;
    double sums[5];
    CK(c, cudaMemcpyAsync(sums, sums_ptr(c), sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (lbm_status s = check_status(c)) return s;
    return finish_residual(c, sums, r, total_energy);
}

size_t lbm_state_bytes(const lbm_ctx *c) {
    if (!c) return 0;
    return sizeof(StateHeader) + 2 * c->buf_bytes;
}

lbm_status lbm_get_state(lbm_ctx *c, void *host, size_t bytes) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!host) return fail(c, LBM_EINVAL, "host is NULL");
    if (bytes < lbm_state_bytes(c)) return fail(c, LBM_EINVAL, "state buffer too small");
    if (!c->initialised) return fail(c, LBM_EINVAL, "lbm_init has not been called");
    DeviceGuard g(c->device);
    StateHeader h{};
    h.magic = STATE_MAGIC;
    h.version = 1;
    h.nx = c->nx;
    h.ny = c->ny;
    h.precision = c->precision;
    h.bc_x = c->bc_x;
    h.bc_y = c->bc_y;
    h.cur = c->cur;
    h.n = c->n;
    h.scale = c->scale;
    h.buf_bytes = c->buf_bytes;
    char *p = (char *)host;
    std::memcpy(p, &h, sizeof(h));
    for (int i = 0; i < 2; ++i)
        CK(c, cudaMemcpyAsync(p + sizeof(h) + i * c->buf_bytes, c->buf[i], c->buf_bytes,
                              cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *c, const void *host, size_t bytes) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (!host) return fail(c, LBM_EINVAL, "host is NULL");
    if (bytes < sizeof(StateHeader)) return fail(c, LBM_EINVAL, "state blob too small");
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != STATE_MAGIC || h.version != 1)
        return fail(c, LBM_EINVAL, "not a phonon LBM state blob");
    if (h.nx != c->nx || h.ny != c->ny || h.precision != c->precision || h.bc_x != c->bc_x ||
        h.bc_y != c->bc_y || h.buf_bytes != c->buf_bytes || (h.cur != 0 && h.cur != 1) ||
        h.n < 0 || !(h.scale > 0.0))
        return fail(c, LBM_EINVAL, "state blob does not match this context");
    if (bytes < lbm_state_bytes(c)) return fail(c, LBM_EINVAL, "state blob truncated");
    DeviceGuard g(c->device);
    const char *p = (const char *)host;
    for (int i = 0; i < 2; ++i)
        CK(c, cudaMemcpyAsync(c->buf[i], p + sizeof(h) + i * c->buf_bytes, c->buf_bytes,
                              cudaMemcpyHostToDevice, c->stream));
    // a restored state starts with a clear status word (no earlier time-out)
    if (c->aux) CK(c, cudaMemsetAsync(status_word(c), 0, sizeof(int), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    c->cur = h.cur;
    c->n = h.n;
    c->scale = h.scale;
    c->have_prev = false;
    c->prev_step = c->n;
    c->initialised = true;
    return LBM_OK;
}

long lbm_step_count(const lbm_ctx *c) { return c ? c->n : -1; }

lbm_status lbm_set_kernel(lbm_ctx *c, int kernel) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (kernel < KERNEL_AUTO || kernel > KERNEL_WAVE)
        return fail(c, LBM_EINVAL, "unknown kernel");
    const int k = resolve_kernel(c, kernel);
    if (k < 0) return fail(c, LBM_EUNSUPPORTED, "kernel cannot run this lattice");
    if (k != c->kernel) {
        DeviceGuard g(c->device);
        drop_graphs(c);
        c->kernel = k;
    }
    return LBM_OK;
}

int lbm_get_kernel(const lbm_ctx *c) { return c ? c->kernel : -1; }

lbm_status lbm_set_rounding(lbm_ctx *c, int rounding) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (rounding != LBM_ROUND_NEAREST && rounding != LBM_ROUND_STOCHASTIC)
        return fail(c, LBM_EINVAL, "unknown rounding");
    if (!has_tile_refs(c->precision) && rounding != LBM_ROUND_NEAREST)
        return fail(c, LBM_EUNSUPPORTED, "stochastic rounding applies to 16-bit storage");
    if (rounding != c->rounding) {
        DeviceGuard g(c->device);
        drop_graphs(c);       // their launches hold the rounding
        c->rounding = rounding;
    }
    return LBM_OK;
}

lbm_status lbm_set_side(lbm_ctx *c, int side, int kind, double value) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (side < LBM_SIDE_LEFT || side > LBM_SIDE_TOP) return fail(c, LBM_EINVAL, "unknown side");
    if (kind < LBM_SIDE_DIFFUSE || kind > LBM_SIDE_HEAT_FLUX)
        return fail(c, LBM_EINVAL, "unknown side treatment");
    if ((side <= LBM_SIDE_RIGHT ? c->bc_x : c->bc_y) != LBM_BC_SIDES)
        return fail(c, LBM_EINVAL, "the side's direction was not created with LBM_BC_SIDES");
    if (!std::isfinite(value)) return fail(c, LBM_EINVAL, "side value is not finite");
    if (kind == LBM_SIDE_DIFFUSE) value = 0.0;
    if (c->initialised && (c->precision == PREC_FP16 || c->precision == PREC_BF16) &&
        side_bound(c, kind, value) * c->scale > 32768.0)
        return fail(c, LBM_EINVAL,
                    "side value too large for the 16-bit storage scale fixed at lbm_init; "
                    "set the sides before lbm_init");
    if (kind != c->side_kind[side] || value != c->side_val[side]) {
        DeviceGuard g(c->device);
        drop_graphs(c);       // captured launches hold the old coefficients
        c->side_kind[side] = kind;
        c->side_val[side] = value;
    }
    return LBM_OK;
}

lbm_status lbm_get_side(const lbm_ctx *c, int side, int *kind, double *value) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (side < LBM_SIDE_LEFT || side > LBM_SIDE_TOP)
        return fail(const_cast<lbm_ctx *>(c), LBM_EINVAL, "unknown side");
    if (kind) *kind = c->side_kind[side];
    if (value) *value = c->side_val[side];
    return LBM_OK;
}

lbm_status lbm_set_staged_config(lbm_ctx *c, int stages, int ctas_per_sm, int consumer_warps,
                                 int l2_evict_first) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (stages < 0 || ctas_per_sm < 0 || consumer_warps < 0)
        return fail(c, LBM_EINVAL, "negative configuration");
    const int cw = consumer_warps > 0 ? consumer_warps : 8;
    if (!staged_supported(c->precision, c->nx, c->ny, cw))
        return fail(c, LBM_EUNSUPPORTED, "nx is not a multiple of the staged tile width");
    DeviceGuard g(c->device);
    StagedPlan p;
    cudaError_t e = staged_plan(c->precision, stages, ctas_per_sm, cw, l2_evict_first, &p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, LBM_EUNSUPPORTED, std::string("staged configuration not possible: ") +
                                             cudaGetErrorString(e));
    }
    drop_graphs(c);
    c->stages_req = stages;
    c->ctas_req = ctas_per_sm;
    c->cw_req = cw;
    c->hint_req = l2_evict_first ? 1 : 0;
    c->plan = p;
    return LBM_OK;
}

lbm_status lbm_get_staged_config(const lbm_ctx *c, int *stages, int *ctas_per_sm,
                                 int *consumer_warps, int *l2_evict_first, int *grid) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (stages) *stages = c->plan.stages;
    if (ctas_per_sm) *ctas_per_sm = c->plan.ctas_per_sm;
    if (consumer_warps) *consumer_warps = c->plan.consumer_warps;
    if (l2_evict_first) *l2_evict_first = c->plan.hint;
    if (grid) *grid = c->plan.grid;
    return LBM_OK;
}

lbm_status lbm_set_graph_chunk(lbm_ctx *c, int steps) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (steps < 0 || steps == 1 || (steps & 1))
        return fail(c, LBM_EINVAL, "graph chunk must be 0 or an even number >= 2");
    DeviceGuard g(c->device);
    drop_graphs(c);
    c->graph_chunk = steps;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx *c, int trial_steps, int *kernel, double *us_per_step) {
    NvtxRange nvtx_("lbm_autotune");
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (trial_steps < 0) return fail(c, LBM_EINVAL, "trial_steps must be >= 0");
    if (trial_steps == 0) trial_steps = 20;
    if (trial_steps & 1) ++trial_steps;       // even: the buffers end where they began
    DeviceGuard g(c->device);
    if (lbm_status s = ensure_scratch(c, false)) return s;   // the status word
    struct Cand { int kernel, stages, cw; };   // wave: stages = steps, cw = segment rows
    Cand cands[16];
    int nc = 0;
    const bool sides = has_sides(c);      // the per-side rules: scalar and vector kernels
    if (c->nx % vector_width(c->precision) == 0) cands[nc++] = {KERNEL_VECTOR, 0, 0};
    else cands[nc++] = {KERNEL_SCALAR, 0, 0};
    for (int cw : {8, 4})
        if (!sides && staged_supported(c->precision, c->nx, c->ny, cw))
            for (int st : {2, 3}) cands[nc++] = {KERNEL_STAGED, st, cw};
    if (resident_ok(c)) cands[nc++] = {KERNEL_RESIDENT, 0, 0};
    if (wave_supported(c->precision, c->nx, c->ny, c->bc_x, c->bc_y) && c->nx >= 128 &&
        c->ny >= 64) {
        if (c->precision == PREC_FP32) {
            for (int ks : {4, 5, 6})
                for (int rows : {128, 256}) cands[nc++] = {KERNEL_WAVE, ks, rows};
        } else {
            for (int ks : {2, 3, 4})
                for (int rows : {128, 256}) cands[nc++] = {KERNEL_WAVE, ks, rows};
        }
    }

    // keep the state: copy both buffers aside when the lattice holds one
    void *saved = nullptr;
    if (c->initialised) {
        CK(c, cudaMallocAsync(&saved, 2 * c->buf_bytes, c->stream));
        for (int i = 0; i < 2; ++i)
            CK(c, cudaMemcpyAsync((char *)saved + i * c->buf_bytes, c->buf[i], c->buf_bytes,
                                  cudaMemcpyDeviceToDevice, c->stream));
    }
    const int old_kernel = c->kernel;
    const StagedPlan old_plan = c->plan;
    const int old_ws = c->wave_steps, old_wr = c->wave_rows;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 0.f;
    int best_i = -1;
    StagedPlan best_plan = c->plan;
    for (int i = 0; i < nc && err == cudaSuccess; ++i) {
        StagedPlan p = c->plan;
        if (cands[i].kernel == KERNEL_STAGED &&
            staged_plan(c->precision, cands[i].stages, 0, cands[i].cw, 0, &p) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        c->kernel = cands[i].kernel;
        c->plan = p;
        long steps_timed = trial_steps;
        if (c->kernel == KERNEL_WAVE) {
            // its point is several steps per launch: time whole launches, an
            // even number (the buffers end where they began)
            c->wave_steps = cands[i].stages;
            c->wave_rows = cands[i].cw;
            int launches = (trial_steps + c->wave_steps - 1) / c->wave_steps;
            launches += launches & 1;
            steps_timed = (long)launches * c->wave_steps;
            for (int s = 0; s < 2 && err == cudaSuccess; ++s)      // warm-up
                err = wave_launch(c, s & 1, c->wave_steps, c->stream);
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
            for (int s = 0; s < launches && err == cudaSuccess; ++s)
                err = wave_launch(c, s & 1, c->wave_steps, c->stream);
        } else if (c->kernel == KERNEL_RESIDENT) {
            // its point is many steps per launch: time one launch of them all
            const Coef<float> kf = make_coef<float>(c);
            float *b0 = (float *)c->buf[0], *b1 = (float *)c->buf[1];
            err = launch_resident(b0, b0, b1, c->nx, c->ny, c->bc_x, c->bc_y, kf, 2, c->rplan,
                                  status_word(c), c->stream);
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
            if (err == cudaSuccess)
                err = launch_resident(b0, b0, b1, c->nx, c->ny, c->bc_x, c->bc_y, kf,
                                      trial_steps, c->rplan, status_word(c), c->stream);
        } else {
            for (int s = 0; s < 2 && err == cudaSuccess; ++s)      // warm-up
                err = dispatch<StepOp>(c, s & 1, c->stream);
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
            for (int s = 0; s < trial_steps && err == cudaSuccess; ++s)
                err = dispatch<StepOp>(c, s & 1, c->stream);
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        ms = ms * (float)trial_steps / (float)steps_timed;      // per trial_steps steps
        if (err == cudaSuccess && (best_i < 0 || ms < best)) {
            best = ms;
            best_i = i;
            best_plan = p;
        }
    }
    c->wave_steps = old_ws;
    c->wave_rows = old_wr;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (saved) {
        for (int i = 0; i < 2 && err == cudaSuccess; ++i)
            err = cudaMemcpyAsync(c->buf[i], (char *)saved + i * c->buf_bytes, c->buf_bytes,
                                  cudaMemcpyDeviceToDevice, c->stream);
        cudaFreeAsync(saved, c->stream);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess || best_i < 0) {
        c->kernel = old_kernel;
        c->plan = old_plan;
        c->wave_steps = old_ws;
        c->wave_rows = old_wr;
        return err != cudaSuccess ? cuda_fail(c, err, "lbm_autotune")
                                  : fail(c, LBM_ECUDA, "no kernel could be timed");
    }
    if (lbm_status s = check_status(c)) return s;
    drop_graphs(c);
    c->kernel = cands[best_i].kernel;
    c->plan = best_plan;
    if (cands[best_i].kernel == KERNEL_WAVE) {
        c->wave_steps = cands[best_i].stages;
        c->wave_rows = cands[best_i].cw;
    }
    if (cands[best_i].kernel == KERNEL_STAGED) {
        c->stages_req = cands[best_i].stages;
        c->ctas_req = 0;
        c->cw_req = cands[best_i].cw;
        c->hint_req = 0;
    }
    if (kernel) *kernel = c->kernel;
    if (us_per_step) *us_per_step = 1000.0 * best / trial_steps;
    return LBM_OK;
}

lbm_status lbm_set_wave_config(lbm_ctx *c, int steps, int rows) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (steps < WAVE_MIN_STEPS || steps > wave_max_steps(c->precision))
        return fail(c, LBM_EINVAL, "steps per launch must be 2..8 (2..4 with 16-bit storage)");
    if (rows < 1) return fail(c, LBM_EINVAL, "rows per segment must be >= 1");
    if (steps != c->wave_steps || rows != c->wave_rows) {
        DeviceGuard g(c->device);
        drop_graphs(c);
        c->wave_steps = steps;
        c->wave_rows = rows;
    }
    return LBM_OK;
}

lbm_status lbm_get_wave_config(const lbm_ctx *c, int *steps, int *rows) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (steps) *steps = c->wave_steps;
    if (rows) *rows = c->wave_rows;
    return LBM_OK;
}

lbm_status lbm_set_launch_timing(lbm_ctx *c, int on) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    DeviceGuard g(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    for (auto &t : c->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->timed.clear();
    for (int i = 0; i < 3; ++i) {
        c->timed_ms[i] = 0.0;
        c->timed_launches[i] = 0;
        c->timed_steps[i] = 0;
    }
    c->timing = on != 0;
    return LBM_OK;
}

lbm_status lbm_launch_time(lbm_ctx *c, int which, double *ms, long long *launches,
                           long long *steps) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    if (which < LBM_TIMED_WAVE || which > LBM_TIMED_RESIDUAL)
        return fail(c, LBM_EINVAL, "unknown launch kind");
    DeviceGuard g(c->device);
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, timed_collect(c));
    if (ms) *ms = c->timed_ms[which];
    if (launches) *launches = c->timed_launches[which];
    if (steps) *steps = c->timed_steps[which];
    return LBM_OK;
}

lbm_status lbm_check_bounded_wait(void *stream, int *gave_up, double *seconds) {
    if (gave_up) *gave_up = 0;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&status, sizeof(int));
    if (err == cudaSuccess) err = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) err = launch_wait_probe(status, s);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    int st = 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(status);
    if (err != cudaSuccess) return cuda_fail(nullptr, err, "lbm_check_bounded_wait");
    if (gave_up) *gave_up = st != 0;
    if (seconds) *seconds = ms / 1e3;
    return LBM_OK;
}

lbm_status lbm_probe_resident_wait(lbm_ctx *c) {
    if (!c) return fail(nullptr, LBM_EINVAL, "ctx is NULL");
    DeviceGuard g(c->device);
    if (lbm_status s = ensure_scratch(c, false)) return s;
    CK(c, launch_resident_wait_probe(status_word(c), c->stream));
    return LBM_OK;
}

long long lbm_kernel_launches(const lbm_ctx *c) { return c ? c->launches : -1; }

double lbm_storage_scale(const lbm_ctx *c) { return c ? c->scale : 0.0; }

const char *lbm_last_error(const lbm_ctx *c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

}  // extern "C"
