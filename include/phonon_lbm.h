/*
 * phonon_lbm.h - C-ABI of the GB300 (sm_103a) phonon lattice Boltzmann solver.
 *
 * The solver advances the lattice Boltzmann equation of Guo & Wang for the
 * phonon Boltzmann equation under Callaway's dual relaxation model
 * (arXiv 2010.01847, Section 2), on a 2-D D2Q8 lattice:
 *
 *   e_i(x + c_i, t + 1) - e_i(x, t) = (e_i^eq - e_i)/tau + S_i        (Eq. 13)
 *   e_i^eq = w_i e + 5 a_i (c_i . q) / 3                              (Eq. 15)
 *   S_i    = -(1 - 1/(2 tau)) 5 a_i (c_i . q) / (3 tau_r)             (Eq. 16)
 *   e = sum_i e_i (Eq. 53),  q = 2 tau_r/(2 tau_r + 1) sum_i c_i e_i  (Eq. 54)
 *   tau = tau_C + 1/2, 1/tau_C = 1/tau_N + 1/tau_R, tau_r = tau_R     (Eq. 49)
 *
 * with w_i, a_i of Eqs. 17-18, in lattice units (dx = dt = c = 1, so
 * v_g = sqrt(5/3) by Eq. 48).  Directions i = 0..7 are the paper's 1..8:
 * (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *
 * Boundaries (Section 2.5): periodic wrap; the periodic temperature-gradient
 * condition along x (Eqs. 59-60: populations crossing the x seam from
 * x = nx-1 to x = 0 gain w_i delta_e, those crossing back lose it); diffuse
 * adiabatic walls on the rows y = 0 and y = ny-1 (Eq. 58: the unknown
 * populations of a wall node are w_i / (5/18) times the sum of its incident
 * ones); and non-periodic directions whose two sides each carry their own
 * treatment (lbm_set_side): diffuse adiabatic (Eq. 58), isothermal (Eq. 55)
 * or an incident heat flux (Eqs. 56-57).  Boundaries sit on the boundary
 * nodes; they act right after streaming; boundary nodes then collide like
 * every other node.
 *
 * STATE CONTRACT.  "The state at step n" is the set of populations after
 * streaming and boundary treatment of step n, before collision.  lbm_init
 * sets step 0 to the equilibrium of Eq. 15; lbm_moments and lbm_residual
 * report e and q of the state at the current step.
 *
 * Conventions for every call:
 *   - Every call returns an lbm_status; nothing throws across the ABI.  The
 *     text of the last failure is lbm_last_error(ctx) (ctx may be NULL for a
 *     failed lbm_create).
 *   - Arguments are checked before any work is queued.
 *   - Host arrays are row-major [ny][nx], index y*nx + x, float64.
 *   - Device pointers are CUDA device addresses on the context's device.
 *   - Calls queue work on the context's stream.  "async" calls return once
 *     the work is queued; a fault inside a kernel is reported by the next
 *     call that synchronises (lbm_sync, lbm_moments, lbm_residual, ...).
 *   - A context is not thread-safe; one host thread drives it at a time.
 */
#ifndef PHONON_LBM_H
#define PHONON_LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,        /* an argument is out of range or NULL           */
    LBM_ENOMEM = 2,        /* a device allocation failed                    */
    LBM_ECUDA = 3,         /* a CUDA call or kernel failed                  */
    LBM_ENONFINITE = 4,    /* the state holds NaN or Inf                    */
    LBM_ETIMEOUT = 5,      /* a bounded device-side wait gave up            */
    LBM_EUNSUPPORTED = 6   /* a valid request this build does not support   */
} lbm_status;

typedef enum {
    LBM_BC_PERIODIC = 0,            /* plain wrap                              */
    LBM_BC_PERIODIC_GRADIENT = 1,   /* Eqs. 59-60; x direction only            */
    LBM_BC_DIFFUSE_WALLS = 2,       /* Eq. 58 on rows 0 and ny-1; y only       */
    LBM_BC_SIDES = 3                /* not periodic: each of the two sides has */
                                    /* its own treatment (lbm_set_side), by    */
                                    /* default diffuse adiabatic; x or y       */
} lbm_bc;

/* The four sides of the lattice (external normals (-1,0), (1,0), (0,-1),
 * (0,1)): the nodes x = 0, x = nx-1, y = 0 and y = ny-1. */
typedef enum {
    LBM_SIDE_LEFT = 0,
    LBM_SIDE_RIGHT = 1,
    LBM_SIDE_BOTTOM = 2,
    LBM_SIDE_TOP = 3
} lbm_side;

/* Treatments of a side of an LBM_BC_SIDES direction (Section 2.5).  With
 * n the side's external normal and kappa = 2 tau_r / (2 tau_r + 1):
 *   LBM_SIDE_DIFFUSE     Eq. 58: the unknown populations (c_i . n < 0) are
 *                        w_i / (5/18) times the sum of the incident ones
 *                        (c_i . n > 0); no energy crosses the side.
 *   LBM_SIDE_ISOTHERMAL  Eq. 55: every population of the node is set to
 *                        w_i e_s, the equilibrium at rest at the side's
 *                        energy density e_s (= C_V T_s).
 *   LBM_SIDE_HEAT_FLUX   Eq. 57: the unknown populations are w_i / (5/18)
 *                        times (sum of the incident ones + q_0 / kappa), so
 *                        that -kappa sum_i (c_i . n) e_i = q_0 (Eq. 56): q_0
 *                        is the flux entering the lattice through the side.
 * A node on two sides (a corner) takes the isothermal treatment of the
 * first isothermal side in the order left, right, bottom, top.  A corner
 * between a LBM_BC_SIDES x side and a y side (walls or a side) with no
 * isothermal side among them has no treatment in the scheme: calls that
 * advance or read such a lattice return LBM_EUNSUPPORTED. */
typedef enum {
    LBM_SIDE_DIFFUSE = 0,
    LBM_SIDE_ISOTHERMAL = 1,
    LBM_SIDE_HEAT_FLUX = 2
} lbm_side_kind;

/* How the populations are stored in device memory.  All but LBM_FP64 store
 * the deviation d_i = s (e_i - w_i e_ref) from the equilibrium at rest at the
 * reference energy e_ref, with s = 1 for LBM_FP32 and a power of two chosen
 * at lbm_init for the 16-bit kinds (so the largest |d_i| sits near 2^12).
 * Collision arithmetic is FP32 for the FP32/FP16/BF16 kinds and FP64 for
 * LBM_FP64 (which also stores deviations, in double).  The FP32 collision has
 * a fixed operation order (each operation rounds once, no contraction left
 * to the compiler), so every kernel kind gives the same bits. */
typedef enum {
    LBM_FP32 = 0,
    LBM_FP16_DEV = 1,
    LBM_BF16_DEV = 2,
    LBM_FP64 = 3
} lbm_precision;

/* Which stream-collide kernel lbm_step launches. */
typedef enum {
    LBM_KERNEL_AUTO = 0,     /* up to 16384 nodes: resident for LBM_FP32,     */
                             /* scalar for LBM_FP64; from 2^24 nodes (nx >=   */
                             /* 256) wave where it applies (FP32: 5 steps     */
                             /* per launch, 128-row segments; 16-bit: 4 and   */
                             /* 256); else                                    */
                             /* vector when nx allows, else scalar            */
                             /* (lbm_autotune times the candidates)           */
    LBM_KERNEL_SCALAR = 1,   /* one thread per node; any nx                   */
    LBM_KERNEL_VECTOR = 2,   /* 16-byte vectors along x; nx % (16/size) == 0  */
    LBM_KERNEL_STAGED = 3,   /* bulk asynchronous copies (TMA engine) of row  */
                             /* (not for lattices with LBM_BC_SIDES)          */
                             /* segments into a shared-memory ring; needs nx  */
                             /* a multiple of the tile width (4096/size with  */
                             /* the default shape)                            */
    LBM_KERNEL_RESIDENT = 4, /* LBM_FP32 lattices small enough that both      */
                             /* population buffers fit in the shared memory   */
                             /* of one thread-block cluster (up to 16 CTAs,   */
                             /* ~3.6 MB: 201 x 201 fits): lbm_step(n) is one  */
                             /* launch of n steps, slabs exchanged through    */
                             /* distributed shared memory; same results bit   */
                             /* for bit.  lbm_set_kernel returns              */
                             /* LBM_EUNSUPPORTED when the lattice does not    */
                             /* fit or no cluster can be resident             */
    LBM_KERNEL_WAVE = 5      /* several steps per launch (temporal blocking): */
                             /* each warp advances a 64-column strip of a     */
                             /* segment of rows K levels in registers         */
                             /* (lbm_set_wave_config), reading and writing    */
                             /* the planes once per K steps.  LBM_FP32: nx    */
                             /* even, same results bit for bit.  LBM_FP16_DEV */
                             /* / LBM_BF16_DEV: nx % 8 == 0, K <= 4; levels   */
                             /* in FP32, stored (rounded to 16 bits) once per */
                             /* launch, so not the bits of single 16-bit      */
                             /* steps.  x periodic (with or without the       */
                             /* gradient), y periodic or walled; else         */
                             /* LBM_EUNSUPPORTED.  lbm_step(n) ends with one  */
                             /* single step (vector kernel, else scalar),     */
                             /* which the read-outs need; lbm_step_residual(n)*/
                             /* runs n - 1 steps in multi-step launches and   */
                             /* its residual step                             */
} lbm_kernel;

typedef struct {
    int nx;                  /* nodes along x (>= 1)                           */
    int ny;                  /* nodes along y (>= 1; >= 2 with walls)          */
} lbm_grid;

typedef struct {
    int x;                   /* LBM_BC_PERIODIC, _PERIODIC_GRADIENT or _SIDES  */
    int y;                   /* LBM_BC_PERIODIC, _DIFFUSE_WALLS or _SIDES      */
    double delta_e;          /* e_h - e_c of Eqs. 59-60 across one x period    */
} lbm_boundary;

/* Eq. 48 in lattice units: tau_X = Kn_X * length * sqrt(3/5), the relaxation
 * time (in steps) of Knudsen number kn over a length of `length` cells. */
double lbm_tau_from_kn(double kn, double length);

/* Bytes of ONE population buffer (8 planes of ny*nx) for lbm_create_ex. */
size_t lbm_population_bytes(lbm_grid grid, lbm_precision precision);

/* Create a solver for a grid, relaxation times in lattice steps (tau_N and
 * tau_R > 0, INFINITY allowed for either but not both; Section 2.1 and
 * Eq. 49), boundaries and storage kind.  e_ref is the reference energy of the
 * deviation storage (any finite value; the results do not depend on it up to
 * rounding).  stream is a cudaStream_t (NULL = legacy default stream) on the
 * current device, which the context remembers.
 * Allocates two population buffers with cudaMalloc; freed by lbm_destroy.
 * The sides of LBM_BC_SIDES directions start diffuse (Eq. 58).
 * Errors: EINVAL (NULL out, grid too small, tau <= 1/2, tau_R <= 0, bad
 * enum), EUNSUPPORTED (gradient on y, walls on x), ENOMEM, ECUDA. */
lbm_status lbm_create(lbm_grid grid, double tau_N, double tau_R,
                      lbm_boundary bc, lbm_precision precision, double e_ref,
                      void *stream, lbm_ctx **out);

/* As lbm_create, but the caller supplies the two population buffers
 * (device pointers, 256-byte aligned, each at least
 * lbm_population_bytes(grid, precision) bytes).  They stay owned by the
 * caller and must outlive the context.  Scratch for moments and residuals is
 * still allocated by the library on first use. */
lbm_status lbm_create_ex(lbm_grid grid, double tau_N, double tau_R,
                         lbm_boundary bc, lbm_precision precision,
                         double e_ref, void *stream, void *buf_a, void *buf_b,
                         size_t buf_bytes, lbm_ctx **out);

/* Free everything the context allocated (never caller-owned buffers).
 * Synchronises the context's stream first.  NULL is accepted. */
void lbm_destroy(lbm_ctx *ctx);

/* Set step 0 to e_i = e_i^eq(e, q) (Eq. 15) from HOST fields e, qx, qy
 * ([ny][nx] float64; qx or qy may be NULL for zero).  Resets the step count
 * and the residual history.  Synchronous.  Errors: EINVAL (NULL ctx or e,
 * non-finite input), ENOMEM, ECUDA. */
lbm_status lbm_init(lbm_ctx *ctx, const double *e, const double *qx,
                    const double *qy);

/* As lbm_init with DEVICE fields (qx, qy may be NULL).  Synchronises once to
 * read the largest deviation for the 16-bit scale. */
lbm_status lbm_init_device(lbm_ctx *ctx, const double *e, const double *qx,
                           const double *qy);

/* Advance n >= 0 steps (Eq. 13 with the boundaries above).  Async; long runs
 * replay a CUDA graph of a fixed chunk of steps.  Errors: EINVAL (n < 0,
 * not initialised), ECUDA (launch failure). */
lbm_status lbm_step(lbm_ctx *ctx, long n);

/* Wait for the context's stream; ECUDA if a queued kernel failed, ETIMEOUT
 * if a bounded device-side wait of the staged kernel gave up. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* e (Eq. 53) and q (Eq. 54) of the state at the current step, into HOST
 * arrays [ny][nx] float64 (any of the three may be NULL).  Synchronous. */
lbm_status lbm_moments(lbm_ctx *ctx, double *e, double *qx, double *qy);

/* Same into DEVICE arrays of ny*nx float64 (any may be NULL).  Async. */
lbm_status lbm_moments_device(lbm_ctx *ctx, double *e, double *qx,
                              double *qy);

/* The 8 populations e_i (not deviations) of the state at the current step,
 * as float64 HOST array [8][ny][nx].  Synchronous. */
lbm_status lbm_populations(lbm_ctx *ctx, double *f);

/* Convergence residual and total energy, summed in FP64 on the device
 * (per-node e and q formed in the compute precision).
 *   r = ||(e, q)^n - (e, q)^m||_2 / ((n - m) ||(e - mean(e), q)^n||_2)
 * where m is the step of the previous lbm_residual call since lbm_init
 * (r = +INFINITY on the first call or when n == m), and
 *   total_energy = sum over nodes of e (Eq. 53).
 * Either output may be NULL.  Synchronous.  Errors: ENONFINITE when any
 * e or q is NaN/Inf (outputs still written), ETIMEOUT when a bounded wait of
 * the staged kernel gave up since lbm_init, ECUDA. */
lbm_status lbm_residual(lbm_ctx *ctx, double *r, double *total_energy);

/* Advance n >= 0 steps and return r and total_energy of the state at the
 * final step, exactly as lbm_step(n) followed by lbm_residual would (same
 * history, same definitions), but with the residual sums reduced inside the
 * last step's stream-collide launch instead of a separate pass over the
 * lattice.  Per-node moments are formed in the compute precision and summed
 * in FP64.  n = 0 is lbm_residual.  Synchronous.  Errors as lbm_step and
 * lbm_residual. */
lbm_status lbm_step_residual(lbm_ctx *ctx, long n, double *r, double *total_energy);

/* Checkpoint: an opaque host blob of lbm_state_bytes(ctx) bytes holding the
 * raw population buffers, the step count and the storage scale.
 * lbm_set_state restores it into a context with the same grid, boundary
 * kinds and storage kind; continuing gives bit-identical results. */
size_t lbm_state_bytes(const lbm_ctx *ctx);
lbm_status lbm_get_state(lbm_ctx *ctx, void *host, size_t bytes);
lbm_status lbm_set_state(lbm_ctx *ctx, const void *host, size_t bytes);

/* Steps taken since lbm_init (or restored by lbm_set_state). */
long lbm_step_count(const lbm_ctx *ctx);

/* Choose the stream-collide kernel (LBM_KERNEL_*).  EUNSUPPORTED when the
 * kernel cannot run this lattice (e.g. VECTOR with a ragged nx). */
lbm_status lbm_set_kernel(lbm_ctx *ctx, int kernel);

/* The kernel lbm_step will launch (never LBM_KERNEL_AUTO). */
int lbm_get_kernel(const lbm_ctx *ctx);

/* Rounding of 16-bit storage (FP16 / BF16 deviations; no counterpart in the
 * paper, which states no precision).  LBM_ROUND_NEAREST (the default) rounds
 * every stored population to nearest even.  LBM_ROUND_STOCHASTIC rounds up
 * with probability equal to the dropped fraction of the value, so the
 * rounding error is zero on average and the errors of a slowly varying
 * field add like a random walk over many steps instead of building up; the
 * random bits are a hash of the node pair, the plane and the two values, so
 * a run is deterministic and every kernel stores the same bits.  It costs
 * instructions (about a third more in the node-pair kernel); round to
 * nearest converges to an exact fixed point at steady state, stochastic
 * rounding to within its noise.  Drops the context's captured graphs.
 * Errors: EINVAL (NULL, unknown mode), EUNSUPPORTED (stochastic with FP32 or
 * FP64 storage). */
typedef enum { LBM_ROUND_NEAREST = 0, LBM_ROUND_STOCHASTIC = 1 } lbm_rounding;
lbm_status lbm_set_rounding(lbm_ctx *ctx, int rounding);

/* Set the treatment of one side of an LBM_BC_SIDES direction (Section 2.5;
 * see lbm_side_kind).  side: LBM_SIDE_*; kind: LBM_SIDE_*; value: e_s (the
 * side's energy density, same units as e) for ISOTHERMAL, q_0 (the heat
 * flux entering through the side, lattice units) for HEAT_FLUX, ignored for
 * DIFFUSE.  Takes effect from the next step; the state is kept, so a
 * treatment can be switched between steps (the heat pulse of Section 3.4:
 * HEAT_FLUX for the pulse, then DIFFUSE).  Side values do not enter the
 * checkpoint of lbm_get_state.  With 16-bit storage, set the sides before
 * lbm_init, which sizes the storage scale for them too.
 * Errors: EINVAL (NULL ctx, bad side or kind, the side's direction is not
 * LBM_BC_SIDES, non-finite value, or a value too large for the 16-bit
 * scale already fixed by lbm_init). */
lbm_status lbm_set_side(lbm_ctx *ctx, int side, int kind, double value);

/* The treatment and value of a side (kind and value may be NULL).
 * Errors: EINVAL (NULL ctx, bad side). */
lbm_status lbm_get_side(const lbm_ctx *ctx, int side, int *kind, double *value);

/* Launch shape of the staged kernel; results do not depend on it.
 *   stages          shared-memory ring depth, 2..6 (0 = default 2)
 *   ctas_per_sm     persistent CTAs per SM (0 = as many as fit)
 *   consumer_warps  4 or 8 (0 = 8): tile width 32 x consumer_warps x
 *                   (16 / element size) nodes; nx must be a multiple of it
 *   l2_evict_first  nonzero: the bulk loads carry an L2 evict-first policy
 * EUNSUPPORTED when the shape cannot be launched for this lattice/device. */
lbm_status lbm_set_staged_config(lbm_ctx *ctx, int stages, int ctas_per_sm,
                                 int consumer_warps, int l2_evict_first);

/* The staged kernel's current shape and persistent grid size (any output
 * may be NULL). */
lbm_status lbm_get_staged_config(const lbm_ctx *ctx, int *stages, int *ctas_per_sm,
                                 int *consumer_warps, int *l2_evict_first, int *grid);

/* Autotuner: times every stream-collide kernel and staged shape that can
 * run this lattice (vector or scalar; staged with 2 or 3 stages and 8 or 4
 * consumer warps; cluster-resident; the multi-step kernel with 4, 5 or 6
 * steps per launch (2, 3 or 4 with 16-bit storage) and segments of 128 or
 * 256 rows, on lattices of at least 128 x 64 nodes), trial_steps steps each
 * (0 = 20) after 2 warm-up steps,
 * on the context's stream, and keeps the fastest for later lbm_step calls.
 * The timings run on the context's own buffers; when the context holds a
 * state (after lbm_init) both buffers are first copied to a temporary
 * device allocation (2 x lbm_population_bytes) and restored afterwards, so
 * the state and the step count are unchanged.  Outputs (may be NULL): the
 * chosen LBM_KERNEL_* and its mean time per step in microseconds.
 * Synchronous. */
lbm_status lbm_autotune(lbm_ctx *ctx, int trial_steps, int *kernel, double *us_per_step);

/* Steps per captured CUDA graph chunk (even, >= 2), or 0 to launch every
 * step directly.  Default 64.  With LBM_KERNEL_WAVE a graph holds an even
 * number of multi-step launches of about this many steps. */
lbm_status lbm_set_graph_chunk(lbm_ctx *ctx, int steps);

/* Shape of the multi-step kernel (LBM_KERNEL_WAVE): `steps` time steps per
 * launch (2..8; 2..4 with 16-bit storage) and strips of `rows` rows (>= 1;
 * clipped to ny).  A launch
 * reads and writes the planes once: 64 B per node per `steps` steps, plus
 * the 2 x steps rows of overlap each segment reads.  Each warp keeps about
 * 27 registers per step level (steps = 4: 158 per thread).  Defaults 4 and
 * 128; lbm_autotune sets both.  EINVAL out of range. */
lbm_status lbm_set_wave_config(lbm_ctx *ctx, int steps, int rows);
lbm_status lbm_get_wave_config(const lbm_ctx *ctx, int *steps, int *rows);

/* Launch timing (no counterpart in the paper).  While on, lbm_step and
 * lbm_step_residual bracket every stream-collide launch with a pair of CUDA
 * events on the context's stream and launch without graphs.  Turning it on
 * or off synchronises the stream and clears the totals.  lbm_launch_time
 * synchronises and returns, for one kind of launch, the summed event time
 * in milliseconds, the number of launches and the time steps they advanced
 * since timing was turned on (outputs may be NULL): */
typedef enum {
    LBM_TIMED_WAVE = 0,      /* multi-step launches (LBM_KERNEL_WAVE)          */
    LBM_TIMED_SINGLE = 1,    /* single-step launches                           */
    LBM_TIMED_RESIDUAL = 2   /* the step of lbm_step_residual (with its sums)  */
} lbm_timed;
lbm_status lbm_set_launch_timing(lbm_ctx *ctx, int on);
lbm_status lbm_launch_time(lbm_ctx *ctx, int which, double *ms, long long *launches,
                           long long *steps);

/* Number of stream-collide kernel launches queued since lbm_init. */
long long lbm_kernel_launches(const lbm_ctx *ctx);

/* The storage scale s of the deviation (1 for FP32/FP64). */
double lbm_storage_scale(const lbm_ctx *ctx);

/* Text of the last failure on this context (or of the last failed
 * lbm_create when ctx is NULL).  Never NULL; valid until the next call. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* ---- Batched solver ------------------------------------------------------
 * Many independent lattices ("instances", e.g. channels of different width
 * and Knudsen numbers) advanced together: every lbm_batch step is ONE
 * persistent kernel launch over a list of work items (instance, run of
 * 16-byte vectors) of all running instances, with each instance's own
 * coefficients (same scheme and boundaries as a single context).  The
 * steady-state solve replays a captured CUDA graph per check window and
 * retires converged instances on the device's work list.  Batching has no
 * counterpart in the paper: each instance advances exactly by the scheme of
 * Section 2 (Eq. 13 with Eqs. 15-16, 53-54, walls of Eq. 58, seam of
 * Eqs. 59-60), bit-identical to a single context of the same instance. */
typedef struct {
    int nx, ny;              /* nx a positive multiple of 16 / element size    */
    double tau_N, tau_R;     /* lattice steps, as lbm_create                   */
    lbm_boundary bc;         /* as lbm_create                                  */
} lbm_instance;

typedef struct lbm_batch lbm_batch;

/* Create a batch of `count` instances sharing a storage kind, reference
 * energy and stream.  Allocates two packed population buffers, the residual
 * history and the work list.  Errors: EINVAL / EUNSUPPORTED per instance
 * (text names the instance), ENOMEM, ECUDA. */
lbm_status lbm_batch_create(const lbm_instance *inst, int count, lbm_precision precision,
                            double e_ref, void *stream, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *batch);

/* Step 0 of every instance (Eq. 15) from HOST fields concatenated in
 * instance order (instance i: ny_i*nx_i values, row-major).  e NULL = e_ref
 * everywhere (the cold start); qx/qy NULL = 0.  Resets step counts, residual
 * history and retirement (every instance runs again).  Synchronous. */
lbm_status lbm_batch_init(lbm_batch *batch, const double *e, const double *qx,
                          const double *qy);

/* Advance every running instance n steps (n launches).  Async. */
lbm_status lbm_batch_step(lbm_batch *batch, long n);

/* Residual (definitions of lbm_residual, history per instance) and total
 * energy of every running instance; arrays of `count` (either may be NULL;
 * retired instances keep their last residual, energy left untouched).
 * Needs at least one step since lbm_batch_init (EUNSUPPORTED otherwise).
 * Synchronous.  ENONFINITE when an instance holds NaN/Inf. */
lbm_status lbm_batch_residuals(lbm_batch *batch, double *r, double *energy);

/* Run to steady state: windows of check_every (even, >= 2) steps, the last
 * step of each reducing every running instance's residual inside its
 * launch; an instance retires once r < tol on two consecutive checks, or
 * when it reaches max_steps.  Outputs (arrays of `count`, may be NULL): the
 * steps each instance ran and its last residual.  Synchronous.  ENONFINITE
 * when an instance became non-finite (it is retired, r = NaN). */
lbm_status lbm_batch_solve(lbm_batch *batch, double tol, int check_every, long max_steps,
                           long *steps, double *r);

/* e and q of instance i's current state into HOST arrays [ny_i][nx_i]
 * (any may be NULL).  Synchronous. */
lbm_status lbm_batch_moments(lbm_batch *batch, int i, double *e, double *qx, double *qy);

/* Work schedule: threads per work item (128, 256 or 512: tile of
 * threads x 16-byte vectors of one instance) and persistent CTAs per SM
 * (0 = as many as fit).  Results do not depend on it. */
lbm_status lbm_batch_set_schedule(lbm_batch *batch, int threads_per_item, int ctas_per_sm);
lbm_status lbm_batch_get_schedule(const lbm_batch *batch, int *threads_per_item,
                                  int *ctas_per_sm, int *grid);

/* Multi-step launches for the batch (LBM_FP32 storage, every nx even):
 * the plain steps of lbm_batch_step and of each lbm_batch_solve window run
 * `steps` (2..8) time steps per launch, each warp advancing a strip of 64
 * columns and `rows` rows of one instance in registers (the kernel of
 * LBM_KERNEL_WAVE, with the instance's coefficients); results bit-identical
 * to single steps.  steps = 0 (the default): one step per launch.
 * lbm_batch_step(n) ends with a single step (the read-outs pull from the
 * buffer the last step read); a solve window ends with its residual step.
 * EINVAL out of range; EUNSUPPORTED for other storage or an odd nx. */
lbm_status lbm_batch_set_wave(lbm_batch *batch, int steps, int rows);
lbm_status lbm_batch_get_wave(const lbm_batch *batch, int *steps, int *rows);

/* Autotuner: times every schedule above (trial_steps steps each, 0 = 10)
 * on the initialised batch and, with LBM_FP32 storage, multi-step launches
 * of 3, 4 or 5 steps with segments of 64 or 128 rows; keeps the fastest per
 * step (us_per_step).  The state is copied aside (2 x population bytes of
 * temporary device memory) and restored.  Synchronous. */
lbm_status lbm_batch_autotune(lbm_batch *batch, int trial_steps, double *us_per_step);

/* Normalised steady profiles of every instance (all need the periodic
 * temperature gradient with delta_e != 0 and a finite tau_R), into a DEVICE
 * float array [count][512]: entries 0..255 are Q(Y) = q_x / q_F at
 * Y = j/255 across the channel (row means, linear interpolation), with the
 * Fourier flux q_F = (5/9) tau_R delta_e / nx (Eqs. 59-60 fix the slope
 * |de/dx| = delta_e / nx); entries 256..511 are E(Y) = (row mean of
 * e + delta_e (x - (nx-1)/2) / nx - e_ref) nx / delta_e, in units of the
 * drop per cell.  Both are set by the gradient alone, so they do not depend
 * on the channel's length.  Synchronous. */
lbm_status lbm_batch_profiles(lbm_batch *batch, float *out);

/* Step 0 of every instance from DEVICE profiles in the layout of
 * lbm_batch_profiles (the learned warm start): q_x = Q(Y) q_F, q_y = 0,
 * e = e_ref + (delta_e / nx) (E(Y) - <E> - (x - (nx-1)/2)), then Eq. 15, where
 * <E> is the row mean of E: a channel conserves its total energy, so the
 * start keeps the cold start's mean energy and reaches the same steady
 * state.  FP32 or FP64 storage.  Resets steps, history and retirement.
 * Synchronous. */
lbm_status lbm_batch_init_profiles(lbm_batch *batch, const float *profiles);

/* The analytic start, as profiles in the layout of lbm_batch_profiles: Q(Y)
 * from Eq. 68 (the heat flux of the phonon hydrodynamic model across a
 * channel between diffuse walls, over the Fourier flux) with
 * Kn_eff = sqrt(tau_C tau_R v_g^2 / 5) / d and Kn_C = v_g tau_C / d in
 * lattice units (v_g = sqrt(5/3), d = ny - 1), and E(Y) = 0 (e affine in x
 * with the steady slope).  For count instances (walls on y, ny >= 2, finite
 * tau_R; nx and delta_e do not enter) into the DEVICE float array out
 * [count][512]: op 0 writes them, op 1 adds them to out, op -1 subtracts
 * them (a learned correction to the analytic profile is trained on the
 * difference and added back).  stream: cudaStream_t (NULL = legacy
 * default).  Allocates a temporary device copy for op != 0.  Synchronous.
 * Errors (text from lbm_last_error(NULL)): EINVAL, EUNSUPPORTED, ECUDA. */
lbm_status lbm_analytic_profiles(const lbm_instance *inst, int count, float *out, int op,
                                 void *stream);

/* Running (not retired) instances, and the steps instance i has run. */
long lbm_batch_active(const lbm_batch *batch);
long lbm_batch_steps(const lbm_batch *batch, int i);

/* Text of the batch's last failure (of the last failed lbm_batch_create via
 * lbm_last_error(NULL)). */
const char *lbm_batch_last_error(const lbm_batch *batch);

/* ---- Warm-start network ---------------------------------------------------
 * A multilayer perceptron trained on the GPU to map a channel's parameters
 * to its steady profile (the layout of lbm_batch_profiles), so a solve can
 * start near steady state.  Layer l: Z = X W_l^T + b_l with W_l stored
 * [width_{l+1}][width_l] row-major; GELU (x Phi(x)) after every layer but
 * the last.  Products take BF16 operands on the tensor cores with FP32
 * accumulation; parameters, gradients and Adam moments are FP32.  The
 * paper has no network: this is the build's warm-start extension. */
typedef struct lbm_mlp lbm_mlp;

/* widths[0] inputs, widths[n_widths-1] outputs; max_batch rows per call. */
lbm_status lbm_mlp_create(const int *widths, int n_widths, int max_batch, void *stream,
                          lbm_mlp **out);
void lbm_mlp_destroy(lbm_mlp *mlp);
/* Number of FP32 parameters: per layer W_l (row-major) then b_l. */
size_t lbm_mlp_param_count(const lbm_mlp *mlp);
/* Copy parameters from / to HOST (FP32, the layout above); setting them
 * clears the Adam moments.  Synchronous. */
lbm_status lbm_mlp_set_params(lbm_mlp *mlp, const float *host);
lbm_status lbm_mlp_get_params(lbm_mlp *mlp, float *host);
/* y = network(x) for `batch` rows: DEVICE float x [batch][in], y [batch][out].
 * Async. */
lbm_status lbm_mlp_forward(lbm_mlp *mlp, const float *x, int batch, float *y);
/* Mean squared error against DEVICE targets t and, if grads is not NULL, its
 * gradient with respect to every parameter into HOST memory (param_count
 * floats).  Synchronous. */
lbm_status lbm_mlp_loss_grad(lbm_mlp *mlp, const float *x, const float *t, int batch,
                             double *loss, float *grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error;
 * *loss is the loss before the update.  Synchronous. */
lbm_status lbm_mlp_train_step(lbm_mlp *mlp, const float *x, const float *t, int batch,
                              float lr, double *loss);
/* `steps` Adam steps (as lbm_mlp_train_step) on minibatches of `batch` rows
 * drawn from n training pairs, DEVICE float x [n][in] and t [n][out], run
 * entirely on the device: one step (minibatch gather, forward, backward,
 * Adam) is captured once as a CUDA graph and replayed, with no host
 * round trip between steps.  Step s (0-based) draws row j of its minibatch
 * as sample SplitMix64(seed ^ (s batch + j)) mod n (with replacement; all n
 * rows in order when batch >= n) and uses the learning rate
 * lr_final + (lr - lr_final)(1 + cos(pi s / steps)) / 2.  The Adam step
 * count carries over between calls.  loss (HOST, `steps` floats, may be
 * NULL) receives each step's loss before its update.  Allocates the
 * minibatch buffers on the first call and the loss history for the call.
 * Synchronous.  Errors: EINVAL (NULL inputs, n < 1, batch out of range,
 * steps < 0, learning rates <= 0), ENOMEM, ECUDA. */
lbm_status lbm_mlp_train(lbm_mlp *mlp, const float *x, const float *t, int n, int batch,
                         long steps, float lr, float lr_final, unsigned long long seed,
                         float *loss);
const char *lbm_mlp_last_error(const lbm_mlp *mlp);

/* ---- Residual without device allocation ---------------------------------
 * The paper has no counterpart to this call; it serves callers that must not
 * allocate device memory while they run: a host application that reserved
 * the device memory for its own pool at start-up and hands out nothing else,
 * a plugin living inside a framework that owns the allocator, or a timing-
 * critical loop that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the whole device.  Such a caller keeps its own moment fields
 * (for example from lbm_moments_device) and asks for the same quantities
 * lbm_residual returns.
 *
 * Inputs: e, qx, qy = DEVICE arrays of n_nodes float64 (e and q at step n);
 * prev_e, prev_qx, prev_qy = the same at step n - k_steps, or all three NULL
 * (then *r = +INFINITY).  e_ref = any finite reference (subtracted before the
 * sums to keep them accurate; results do not depend on it up to rounding).
 * Outputs (HOST, either may be NULL): r and total_energy with the definitions
 * of lbm_residual.  Work is queued on `stream` (cudaStream_t, NULL = legacy
 * default stream) on the current device; the call synchronises that stream.
 *
 * Memory: allocates nothing.  Its scratch is a fixed device array of
 * 163,880 bytes inside the library, present on every device that loads the
 * library until the process exits.  The first call on each device looks up
 * that array's device address (with that device current) and caches it;
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents: calls that overlap on the GPU
 * (different streams, or threads of one process) race and must be
 * serialised by the caller.
 * Limit: n_nodes <= LBM_NOALLOC_MAX_NODES (4096 x 4096 nodes).
 * Errors (text from lbm_last_error(NULL)): EINVAL (NULL inputs, only some
 * previous fields, n_nodes < 1 or above the limit, non-finite e_ref),
 * ENONFINITE (a field holds NaN/Inf; outputs still written), ECUDA. */
#define LBM_NOALLOC_MAX_NODES 16777216LL
lbm_status lbm_residual_noalloc(const double *e, const double *qx, const double *qy,
                                const double *prev_e, const double *prev_qx,
                                const double *prev_qy, long long n_nodes, double e_ref,
                                long k_steps, void *stream, double *r, double *total_energy);

/* Self-check of the failure path of the staged kernel's waits (no
 * counterpart in the paper).  Every mbarrier wait in the staged kernel is
 * bounded by an iteration count and a clock limit (about 2 s); when it gives
 * up it sets the context's status word, which the next synchronising call
 * reports as LBM_ETIMEOUT, and the CTA drains its copies and exits, so the
 * CUDA context stays usable.  This call runs that same wait, in one thread
 * of one CTA, on a fresh barrier that nothing completes, on `stream`
 * (cudaStream_t, NULL = legacy default) of the current device, and waits
 * for it: *gave_up = 1 when the wait ended by its limit and set the status
 * word, *seconds = the kernel's duration (either pointer may be NULL).
 * Allocates 4 bytes of device memory for the duration of the call.
 * Errors: ECUDA (text from lbm_last_error(NULL)). */
lbm_status lbm_check_bounded_wait(void *stream, int *gave_up, double *seconds);

/* Self-check of the failure path of the cluster-resident kernel's ghost
 * exchange (no counterpart in the paper).  Each CTA of that kernel waits,
 * bounded by an iteration count and a clock limit (about 2 s), for the
 * bytes its neighbours store into its ghost cells; a wait that gives up
 * sets bit 2 of the context's status word, and every CTA of the launch then
 * stops stepping, writes nothing and leaves, so one stalled exchange costs
 * one wait limit per launch.  This call runs that same wait, in one thread
 * of a one-CTA cluster, on a fresh barrier that nothing completes,
 * asynchronously on the context's stream with the context's status word:
 * the next synchronising call on ctx (lbm_sync, lbm_moments, ...) returns
 * LBM_ETIMEOUT naming the cluster-resident kernel.  The context's state is
 * untouched; lbm_init (or lbm_set_state) clears the status word.
 * Errors: EINVAL (NULL ctx), ENOMEM, ECUDA. */
lbm_status lbm_probe_resident_wait(lbm_ctx *ctx);

/* ------------------------------------------------------------------------ *
 * The D1Q2 and D3Q14 lattices (periodic lattices only).
 *
 * Section 2.2 says the scheme extends to the one-dimensional D1Q2 and the
 * three-dimensional D3Q14 lattices without giving their weights.  These
 * calls use the weights the Chapman-Enskog analysis of Section 2.3 requires
 * of a velocity set: sum w_i = 1, sum w_i c_ia c_ib = (5/9) delta_ab, sum
 * h_i c_ia c_ib = delta_ab and an isotropic fourth moment sum h_i c c c c =
 * (1/3)(dd + dd + dd), with e_i^eq = w_i e + h_i c_i . q (Eq. 15) and
 * S_i = -(1 - 1/(2 tau)) h_i c_i . q / tau_r (Eq. 16):
 *   D3Q14: c_i = (+-1,0,0), (0,+-1,0), (0,0,+-1) with w = 1/9, h = 1/3;
 *          (+-1,+-1,+-1) with w = 1/24, h = 1/24.  It recovers Eqs. 6-7 in
 *          three dimensions with the lattice speed c = sqrt(3/5) v_g of
 *          Eq. 48 and tau = tau_C + 1/2 (Eq. 49).
 *   D1Q2:  c_i = +-1, w = h = 1/2.  Two velocities cannot carry the nonlocal
 *          term of Eq. 7: the lattice recovers Eq. 6 and Eq. 7 without it
 *          (the Cattaneo equation), with c = v_g / sqrt(3).
 * Directions (population plane order): D3Q14 +x, -x, +y, -y, +z, -z, then
 * +b, -b for b = (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1); D1Q2 +x, -x.
 * Layout: host arrays [nz][ny][nx] float64 (index (z*ny + y)*nx + x); a
 * flux array holds dim planes (x, then y, then z).  Populations are stored
 * as FP32 or FP64 deviations from w_i e_ref; the state contract, the graph
 * chunks and the error conventions are those of the D2Q8 calls above. */
typedef enum {
    LBM_LATTICE_D1Q2 = 1,
    LBM_LATTICE_D3Q14 = 3
} lbm_lattice;

typedef struct lbm_nd lbm_nd;

/* c / v_g of a lattice (sqrt(3/5) for D3Q14, 1/sqrt(3) for D1Q2; 0 for an
 * unknown lattice): a Knudsen number Kn over L cells gives the relaxation
 * time Kn * L * (c / v_g) in steps. */
double lbm_nd_lattice_speed(int lattice);

/* Create a periodic nx x ny x nz lattice (D1Q2: ny = nz = 1).  tau_N, tau_R
 * as for lbm_create; precision LBM_FP32 or LBM_FP64.  Allocates two
 * population buffers of Q * nx * ny * nz elements.
 * Errors: EINVAL (bad lattice, sizes, tau, e_ref, NULL out), EUNSUPPORTED
 * (16-bit storage), ENOMEM, ECUDA (text from lbm_nd_last_error(NULL)). */
lbm_status lbm_nd_create(int lattice, int nx, int ny, int nz, double tau_N, double tau_R,
                         int precision, double e_ref, void *stream, lbm_nd **out);

/* Step 0 = Eq. 15 from HOST e[n] and q[dim][n] (q may be NULL for zero).
 * Synchronises.  Errors: EINVAL (NULL, non-finite input), ECUDA. */
lbm_status lbm_nd_init(lbm_nd *ctx, const double *e, const double *q);

/* Advance n >= 0 steps (async; 64-step CUDA graphs for long runs). */
lbm_status lbm_nd_step(lbm_nd *ctx, long n);

/* Wait for the queued work. */
lbm_status lbm_nd_sync(lbm_nd *ctx);

/* e[n] and q[dim][n] (HOST, either may be NULL) of the current state
 * (Eqs. 53-54).  Synchronises. */
lbm_status lbm_nd_moments(lbm_nd *ctx, double *e, double *q);

/* Populations e_i of the current state, HOST f[Q][n].  Synchronises. */
lbm_status lbm_nd_populations(lbm_nd *ctx, double *f);

/* Total energy sum e of the current state (FP64 reduction, deterministic).
 * ENONFINITE if the state holds NaN or Inf.  Synchronises. */
lbm_status lbm_nd_energy(lbm_nd *ctx, double *total);

long lbm_nd_step_count(const lbm_nd *ctx);
void lbm_nd_destroy(lbm_nd *ctx);
const char *lbm_nd_last_error(const lbm_nd *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PHONON_LBM_H */
