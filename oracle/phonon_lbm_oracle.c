/*
 * Plain FP64 CPU oracle for the phonon lattice Boltzmann scheme of Guo & Wang,
 * "Lattice Boltzmann scheme for hydrodynamic equation of phonon transport"
 * (arXiv 2010.01847): Callaway dual relaxation, D2Q8 lattice.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * It executes Eq. 13 literally, in the paper's order, for every time step:
 *   1. per node: e (Eq. 53), q (Eq. 54), e_i^eq (Eq. 15), Delta t S_i
 *      (Eq. 16), post-collision e_i + (e_i^eq - e_i)/tau + Delta t S_i
 *      (right-hand side of Eq. 13);
 *   2. push-stream every post-collision population to x + c_i (left-hand side
 *      of Eq. 13), wrapping periodic sides and adding the jump of the periodic
 *      temperature-gradient condition (Eqs. 59-60) on the x seam; populations
 *      that leave through a wall are dropped;
 *   3. overwrite the unknown populations of wall nodes by the diffuse
 *      adiabatic reflection (Eq. 58), or, on sides with their own
 *      treatment, by Eq. 57 (incident heat flux) or Eq. 55 (isothermal).
 * The state "at step n" is the set of populations after stream + boundary of
 * step n, before collision.
 *
 * Lattice units: dx = dt = c = 1, so v_g = sqrt(5/3) (Eq. 48) and a relaxation
 * time tau_X (lattice) = Kn_X * L * sqrt(3/5).
 *
 * Layout: array of structures, f[(y*nx + x)*8 + i], i = 0..7 standing for the
 * paper's directions 1..8 (Eq. 14):
 *   1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 * The order is the one Eqs. 59-60 imply (1,5,8 move right; 3,6,7 move left).
 *
 * Readings where the paper is silent (each fixed the same way for the CUDA
 * path): the tau inside (1 - 1/(2 tau)) of Eq. 16 is the overall tau of
 * Eq. 49; the q entering Eqs. 15-16 is the corrected flux of Eq. 54; walls
 * sit on the boundary nodes; the boundary acts right after streaming and the
 * wall nodes then collide like any other node; the x seam lies between node
 * nx-1 and node 0.
 *
 * Rounding: IEEE FP64, fixed loop order.  Build with -ffp-contract=off so no
 * fused multiply-add changes results between machines.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Boundary kinds (oracle's own numbering).  ORC_SIDES: the direction is not
 * periodic and each of its two sides has its own treatment (below). */
enum { ORC_PERIODIC = 0, ORC_PERIODIC_GRADIENT = 1, ORC_WALLS = 2, ORC_SIDES = 3 };

/* Side treatments (Section 2.5): diffuse adiabatic reflection (Eq. 58),
 * isothermal equilibrium at e_s = C_V T_s (Eq. 55), incident heat flux q_0
 * (Eq. 57).  Sides are numbered left (x = 0), right (x = nx-1), bottom
 * (y = 0), top (y = ny-1). */
enum { ORC_DIFFUSE = 0, ORC_ISOTHERMAL = 1, ORC_HEAT_FLUX = 2 };

/* Eq. 14: lattice velocities in units of c. */
static const int CX[8] = {1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[8] = {0, 1, 0, -1, 1, 1, -1, -1};

/* Eq. 17: weights of the energy part of the equilibrium. */
static double omega_w(int i) { return i < 4 ? 2.0 / 9.0 : 1.0 / 36.0; }

/* Eq. 18: weights of the heat-flux part of the equilibrium and source. */
static double a_w(int i) { return i < 4 ? 1.0 / 5.0 : 1.0 / 20.0; }

static int n_threads = 1;

void orc_set_threads(int n) { n_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return n_threads; }

/* Eq. 48 with dx = c dt = 1: v_g = sqrt(5/3); Kn = v_g tau / L. */
double orc_tau_from_kn(double kn, double length)
{
    return kn * length * sqrt(3.0 / 5.0);
}

/* Scalar set-up.  tau_C from 1/tau_C = 1/tau_N + 1/tau_R (Section 2.1);
 * tau = tau_C/dt + 1/2 (Eq. 49); tau_r = tau_R/dt (Section 2.4).
 * Either relaxation time may be +inf.  out = {tau, tau_r, tau_C}. */
void orc_params(double tau_N, double tau_R, double *out)
{
    double inv_c = 0.0;
    if (!isinf(tau_N)) inv_c += 1.0 / tau_N;
    if (!isinf(tau_R)) inv_c += 1.0 / tau_R;
    double tau_C = 1.0 / inv_c;
    out[0] = tau_C + 0.5;
    out[1] = tau_R;
    out[2] = tau_C;
}

/* Eq. 54 prefactor 2 tau_r / (2 tau_r + 1); equals 1 when tau_r = inf. */
static double flux_factor(double tau_r)
{
    if (isinf(tau_r)) return 1.0;
    return 2.0 * tau_r / (2.0 * tau_r + 1.0);
}

/* Eq. 15: e_i^eq = w_i e + 5 a_i (c_i . q) / (3 c^2). */
void orc_equilibrium(double e, double qx, double qy, double *eeq)
{
    for (int i = 0; i < 8; ++i) {
        double cq = CX[i] * qx + CY[i] * qy;
        eeq[i] = omega_w(i) * e + 5.0 * a_w(i) * cq / 3.0;
    }
}

/* Eq. 16 times dt: dt S_i = -(1 - 1/(2 tau)) 5 a_i (c_i . q) / (3 tau_r c^2).
 * Zero when tau_r = inf. */
void orc_source(double qx, double qy, double tau, double tau_r, double *s)
{
    for (int i = 0; i < 8; ++i) {
        if (isinf(tau_r)) {
            s[i] = 0.0;
            continue;
        }
        double cq = CX[i] * qx + CY[i] * qy;
        s[i] = -(1.0 - 1.0 / (2.0 * tau)) * 5.0 * a_w(i) * cq / (3.0 * tau_r);
    }
}

/* Eq. 53 (e = sum e_i) and Eq. 54 (q = 2 tau_r/(2 tau_r+1) sum c_i e_i). */
void orc_node_moments(const double *f, double tau_r, double *e, double *qx,
                      double *qy)
{
    double s = 0.0, mx = 0.0, my = 0.0;
    for (int i = 0; i < 8; ++i) {
        s += f[i];
        mx += CX[i] * f[i];
        my += CY[i] * f[i];
    }
    double k = flux_factor(tau_r);
    *e = s;
    *qx = k * mx;
    *qy = k * my;
}

/* Right-hand side of Eq. 13 at one node: post_i = f_i + (eeq_i - f_i)/tau
 * + dt S_i, with e, q from the node's own populations (Eqs. 53-54). */
void orc_collide_node(const double *f, double tau, double tau_r, double *post)
{
    double e, qx, qy, eeq[8], s[8];
    orc_node_moments(f, tau_r, &e, &qx, &qy);
    orc_equilibrium(e, qx, qy, eeq);
    orc_source(qx, qy, tau, tau_r, s);
    for (int i = 0; i < 8; ++i)
        post[i] = f[i] + (eeq[i] - f[i]) / tau + s[i];
}

/* Initial state: e_i = e_i^eq(e, q) at every node (Eq. 15).  Inputs are
 * ny*nx row-major fields, index y*nx + x. */
void orc_init(int nx, int ny, const double *e, const double *qx,
              const double *qy, double *f)
{
    for (long s = 0; s < (long)nx * ny; ++s)
        orc_equilibrium(e[s], qx[s], qy[s], f + s * 8);
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Eq. 57 (Eq. 58 when q0 = 0) at one boundary node with external normal
 * (nxo, nyo): the populations leaving the surface into the domain
 * (c . n < 0) are w_i / sum_leaving(w) times the sum of the incident ones
 * (c . n > 0) plus q0/c (2 tau_r + 1)/(2 tau_r). */
static void flux_side(double *g, int nxo, int nyo, double q0, double tau_r)
{
    double w_leave = 0.0, incident = 0.0;
    for (int i = 0; i < 8; ++i) {
        int cn = CX[i] * nxo + CY[i] * nyo;
        if (cn < 0) w_leave += omega_w(i);
        if (cn > 0) incident += g[i];
    }
    double extra = q0 / flux_factor(tau_r);
    for (int i = 0; i < 8; ++i)
        if (CX[i] * nxo + CY[i] * nyo < 0)
            g[i] = omega_w(i) / w_leave * (incident + extra);
}

/* Eq. 55: every population of the node at equilibrium at rest at e_s. */
static void isothermal_node(double *g, double e_s)
{
    for (int i = 0; i < 8; ++i) g[i] = omega_w(i) * e_s;
}

/* Boundary treatment of the sides of ORC_SIDES directions, after
 * streaming.  A node on an isothermal side is set by Eq. 55 (an x side's
 * value first when two isothermal sides meet at a corner); otherwise its
 * y side, then its x side, applies Eq. 57 / Eq. 58 (the paper's cases have
 * no such corner). */
static void sides_pass(int nx, int ny, int bc_x, int bc_y, const int *kind,
                       const double *val, double tau_r, double *f)
{
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int on[4] = {0, 0, 0, 0};
            if (bc_x == ORC_SIDES) { on[0] = x == 0; on[1] = x == nx - 1; }
            if (bc_y == ORC_SIDES) { on[2] = y == 0; on[3] = y == ny - 1; }
            if (!(on[0] || on[1] || on[2] || on[3])) continue;
            double *g = f + ((long)y * nx + x) * 8;
            int iso = -1;
            for (int sd = 0; sd < 4 && iso < 0; ++sd)
                if (on[sd] && kind[sd] == ORC_ISOTHERMAL) iso = sd;
            if (iso >= 0) {
                isothermal_node(g, val[iso]);
                continue;
            }
            static const int order[4] = {2, 3, 0, 1};
            static const int nrm[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
            for (int o = 0; o < 4; ++o) {
                int sd = order[o];
                if (!on[sd]) continue;
                double q0 = kind[sd] == ORC_HEAT_FLUX ? val[sd] : 0.0;
                flux_side(g, nrm[sd][0], nrm[sd][1], q0, tau_r);
            }
        }
    }
}

/* One time step in place: collision, push streaming with periodic wrap and
 * the Eq. 59-60 seam jump, then the boundary treatments.  tmp holds
 * nx*ny*8 doubles of scratch. */
static void one_step(int nx, int ny, int bc_x, int bc_y, double delta_e,
                     const int *kind, const double *val,
                     double tau, double tau_r, double *f, double *tmp)
{
    long n_sites = (long)nx * ny;

    /* 1. collision at every node (Eq. 13 right-hand side), into tmp */
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (long s = 0; s < n_sites; ++s)
        orc_collide_node(f + s * 8, tau, tau_r, tmp + s * 8);

    /* slots that no population streams into stay NaN until the boundary
     * fills them, so a missed boundary treatment cannot pass silently */
    for (long k = 0; k < n_sites * 8; ++k)
        f[k] = NAN;

    /* 2. push streaming: post-collision e_i at x lands at x + c_i */
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const double *src = tmp + ((long)y * nx + x) * 8;
            for (int i = 0; i < 8; ++i) {
                int tx = x + CX[i];
                int ty = y + CY[i];
                double v = src[i];
                if (ty < 0 || ty >= ny) {
                    if (bc_y == ORC_WALLS || bc_y == ORC_SIDES)
                        continue;           /* leaves through the wall */
                    ty = wrap(ty, ny);
                }
                if (tx < 0 || tx >= nx) {
                    if (bc_x == ORC_SIDES)
                        continue;           /* leaves through the side */
                    if (bc_x == ORC_PERIODIC_GRADIENT) {
                        /* Eq. 59: i = 1,5,8 entering on the left gain
                         * w_i (e_h - e_c); Eq. 60: i = 3,6,7 entering on
                         * the right lose it. */
                        if (tx >= nx)
                            v = omega_w(i) * delta_e + v;
                        else
                            v = v - omega_w(i) * delta_e;
                    }
                    tx = wrap(tx, nx);
                }
                f[((long)ty * nx + tx) * 8 + i] = v;
            }
        }
    }

    /* 3. diffuse adiabatic walls, Eq. 58, on the unknowns c_i . n < 0 */
    if (bc_y == ORC_WALLS) {
        for (int side = 0; side < 2; ++side) {
            int y = side == 0 ? 0 : ny - 1;
            int ny_out = side == 0 ? -1 : 1;    /* external normal (0, ny_out) */
            double w_leave = 0.0;
            for (int i = 0; i < 8; ++i)
                if (CY[i] * ny_out < 0) w_leave += omega_w(i);
            for (int x = 0; x < nx; ++x) {
                double *g = f + ((long)y * nx + x) * 8;
                double incident = 0.0;
                for (int i = 0; i < 8; ++i)
                    if (CY[i] * ny_out > 0) incident += g[i];
                for (int i = 0; i < 8; ++i)
                    if (CY[i] * ny_out < 0)
                        g[i] = omega_w(i) / w_leave * incident;
            }
        }
    }

    /* 4. isothermal / heat-flux / diffuse sides, Eqs. 55, 57, 58 */
    if (bc_x == ORC_SIDES || bc_y == ORC_SIDES)
        sides_pass(nx, ny, bc_x, bc_y, kind, val, tau_r, f);
}

/* Advance n_steps time steps.  bc_x: ORC_PERIODIC or ORC_PERIODIC_GRADIENT;
 * bc_y: ORC_PERIODIC or ORC_WALLS.  delta_e = e_h - e_c of Eqs. 59-60.
 * Returns 0, or -1 when the arguments are outside the scheme. */
int orc_run_sides(int nx, int ny, int bc_x, int bc_y, double delta_e,
                  const int *side_kind, const double *side_val,
                  double tau_N, double tau_R, double *f, long n_steps)
{
    if (nx < 1 || ny < 1 || (bc_y == ORC_WALLS && ny < 2)) return -1;
    if (bc_x == ORC_WALLS || bc_y == ORC_PERIODIC_GRADIENT) return -1;
    if ((bc_x == ORC_SIDES && nx < 2) || (bc_y == ORC_SIDES && ny < 2)) return -1;
    static const int diffuse[4] = {0, 0, 0, 0};
    static const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    if (!side_kind) side_kind = diffuse;
    if (!side_val) side_val = zero;
    double p[3];
    orc_params(tau_N, tau_R, p);
    if (!(p[0] > 0.5)) return -1;
    double *tmp = (double *)malloc(sizeof(double) * 8 * (size_t)nx * ny);
    if (!tmp) return -1;
    for (long n = 0; n < n_steps; ++n)
        one_step(nx, ny, bc_x, bc_y, delta_e, side_kind, side_val, p[0], p[1], f, tmp);
    free(tmp);
    return 0;
}

int orc_run(int nx, int ny, int bc_x, int bc_y, double delta_e,
            double tau_N, double tau_R, double *f, long n_steps)
{
    return orc_run_sides(nx, ny, bc_x, bc_y, delta_e, 0, 0, tau_N, tau_R, f, n_steps);
}

/* e, q of every node of a state (Eqs. 53-54). */
void orc_moments(int nx, int ny, double tau_R, const double *f, double *e,
                 double *qx, double *qy)
{
    for (long s = 0; s < (long)nx * ny; ++s)
        orc_node_moments(f + s * 8, tau_R, e + s, qx + s, qy + s);
}
