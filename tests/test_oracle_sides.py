"""Pins of the oracle's side boundary treatments (Section 2.5: isothermal
Eq. 55, heat flux Eqs. 56-57, diffuse Eq. 58 on any side) and of the
continuum solutions of Section 3 that the paper validates them with.

The closed forms in ``oracle.analytic`` are first pinned by properties that
define them (boundary values, the governing equations by finite differences,
energy balance, known Laplace pairs); the oracle is then compared with them
on the paper's cases (Sections 3.1, 3.3 and 3.4) at the accuracy a
first-order scheme reaches on the grids used.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import analytic
from oracle import update_matrix as um

S = oracle.SIDES
DIF, ISO, FLX = oracle.DIFFUSE, oracle.ISOTHERMAL, oracle.HEAT_FLUX
VG = math.sqrt(5.0 / 3.0)        # v_g in lattice units (Eq. 48, c = 1)


def _l1(a, b):
    """Relative L1 error norm of Eqs. 63-64."""
    return np.abs(a - b).sum() / np.abs(b).sum()


# --- the closed forms, pinned by their defining properties -------------------
def test_fourier_transient_solves_heat_equation():
    kn = 1.29e-3
    X = np.linspace(0.0, 1.0, 401)
    h = X[1] - X[0]
    t, dt = 2e5, 50.0
    th, Q = analytic.fourier_transient_1d(X, t, kn)
    thp, _ = analytic.fourier_transient_1d(X, t + dt, kn)
    thm, _ = analytic.fourier_transient_1d(X, t - dt, kn)
    # d Theta / dt* = (Kn_R^2 / 3) d2 Theta / dX2 (Fourier, X = x/d, t* = t/tau_R)
    lhs = (thp - thm) / (2 * dt)
    rhs = kn ** 2 / 3 * (th[2:] - 2 * th[1:-1] + th[:-2]) / h ** 2
    np.testing.assert_allclose(lhs[1:-1], rhs, rtol=2e-4, atol=1e-12)
    # Fourier's law Q = -d Theta / dX, and the boundary values
    np.testing.assert_allclose(Q[1:-1], -(th[2:] - th[:-2]) / (2 * h), rtol=1e-4)
    assert th[0] == pytest.approx(1.0, abs=1e-12) and th[-1] == pytest.approx(0.0, abs=1e-12)
    th_inf, Q_inf = analytic.fourier_transient_1d(X, 1e12, kn)
    np.testing.assert_allclose(th_inf, 1 - X, atol=1e-12)
    np.testing.assert_allclose(Q_inf, 1.0, atol=1e-12)


def test_square_steady_solves_laplace_with_its_boundary_values():
    g = np.linspace(0.0, 1.0, 201)
    Y, X = np.meshgrid(g, g, indexing="ij")
    h = g[1] - g[0]
    th, Qx, Qy = analytic.square_steady(X, Y)
    # Theta = 0 on three sides, dTheta/dY = Q0 = 1 on the top (incident flux)
    np.testing.assert_allclose(th[:, 0], 0.0, atol=1e-12)
    np.testing.assert_allclose(th[:, -1], 0.0, atol=1e-12)
    np.testing.assert_allclose(th[0, :], 0.0, atol=1e-12)
    np.testing.assert_allclose(Qy[-1, 60:141], -1.0, atol=3e-3)
    # Laplace's equation and Q = -grad Theta in the interior
    lap = (th[2:, 1:-1] + th[:-2, 1:-1] + th[1:-1, 2:] + th[1:-1, :-2]
           - 4 * th[1:-1, 1:-1]) / h ** 2
    th_xx = (th[1:-1, 2:] - 2 * th[1:-1, 1:-1] + th[1:-1, :-2]) / h ** 2
    assert np.abs(lap[:-20, 20:-20]).max() < 1e-3 * np.abs(th_xx[:-20, 20:-20]).max()
    np.testing.assert_allclose(Qx[100, 1:-1], -(th[100, 2:] - th[100, :-2]) / (2 * h),
                               atol=2e-4)
    np.testing.assert_allclose(Qy[1:-1, 100], -(th[2:, 100] - th[:-2, 100]) / (2 * h),
                               atol=2e-4)


def test_cross_plane_limits():
    X = np.linspace(0, 1, 11)
    th, Q = analytic.cross_plane(X, 1e-9)           # Fourier limit
    np.testing.assert_allclose(th, 1 - X, atol=1e-8)
    assert Q == pytest.approx(1e-9 / 3, rel=1e-6)
    th, Q = analytic.cross_plane(X, 1e9)            # drift limit
    np.testing.assert_allclose(th, 0.5, atol=1e-8)
    assert Q == pytest.approx(0.25, rel=1e-8)
    th, _ = analytic.cross_plane(X, 1.0)            # symmetric jumps
    np.testing.assert_allclose(th + th[::-1], 1.0, atol=1e-14)


@pytest.mark.parametrize("gamma_t", [3.0, 9.0])
def test_laplace_inverse_known_pairs(gamma_t):
    """Eq. B16 with T_p = t reproduces f(t) up to its aliasing term
    exp(-2 gamma t) f(3 t) (the next one, exp(-4 gamma t) f(5 t), is below
    the tolerance for both gamma t)."""
    pairs = [(lambda s: 1.0 / (s + 1.0), lambda t: math.exp(-t)),
             # unit pulse of length 3, integrated once: a ramp that stops at 3
             (lambda s: (1 - np.exp(-3 * s)) / s ** 2, lambda t: min(t, 3.0))]
    for F, f in pairs:
        for t in (0.5, 2.0, 7.0):
            got = analytic.laplace_inverse(F, t, gamma_t, 20000)
            alias = math.exp(-2 * gamma_t) * f(3 * t)
            assert got == pytest.approx(f(t) + alias, abs=2e-5 * max(1.0, f(t)))


def test_heat_pulse_energy_balance_and_boundary_flux():
    kn_N, kn_R = 1.29e-3, 1.29
    X = np.linspace(0, 1, 2001)
    # Eqs. 77 and 80: after the pulse the mean Theta is Kn_N t_pulse, the
    # terminal rise 0.129 of Section 3.4
    th, _ = analytic.heat_pulse(X, 400.0, kn_N, kn_R, gamma_t=9.0, terms=4000)
    assert np.trapezoid(th, X) == pytest.approx(100 * kn_N, rel=1e-5)
    _, Q = analytic.heat_pulse(np.array([0.0, 1.0]), 50.0, kn_N, kn_R, gamma_t=9.0,
                               terms=4000)
    assert Q[0] == pytest.approx(1.0, abs=1e-4) and Q[1] == pytest.approx(0.0, abs=1e-4)
    _, Q = analytic.heat_pulse(np.array([0.0]), 150.0, kn_N, kn_R, gamma_t=9.0, terms=40000)
    assert Q[0] == pytest.approx(0.0, abs=2e-4)    # slow (1/terms) after the switch-off
    # after the wave has reached the far side and been reflected (t* ~ 1340):
    # still no flux through X = 1 and no energy lost
    X = np.linspace(0, 1, 401)
    th, Q = analytic.heat_pulse(X, 2500.0, kn_N, kn_R, gamma_t=9.0, terms=20000)
    assert np.trapezoid(th, X) == pytest.approx(100 * kn_N, rel=1e-4)
    assert abs(Q[-1]) < 1e-9


# --- the side treatments of the oracle (Eqs. 55-58) ---------------------------
SIDE_CASES = [
    (5, 4, S, oracle.PERIODIC, 0.0, [(ISO, 1.3), (FLX, 0.02), (DIF, 0.0), (DIF, 0.0)]),
    (4, 5, S, S, 0.0, [(ISO, 0.9), (ISO, 1.1), (DIF, 0.0), (FLX, -0.03)]),
    (5, 4, oracle.PERIODIC_GRADIENT, S, 0.3, [(DIF, 0.0), (DIF, 0.0), (FLX, 0.05), (ISO, 1.2)]),
    (4, 4, S, oracle.WALLS, 0.0, [(ISO, 1.05), (ISO, 0.95), (DIF, 0.0), (DIF, 0.0)]),
    (3, 5, oracle.PERIODIC, S, 0.0, [(DIF, 0.0), (DIF, 0.0), (FLX, 0.01), (FLX, -0.02)]),
]


@pytest.mark.parametrize("nx,ny,bc_x,bc_y,de,sides", SIDE_CASES)
def test_brute_force_matrix_with_sides(nx, ny, bc_x, bc_y, de, sides):
    tau_N, tau_R = 0.9, 2.1
    p = oracle.params(tau_N, tau_R)
    rng = np.random.default_rng(11)
    f0 = rng.uniform(0.0, 0.3, (ny, nx, 8))
    lat = oracle.Lattice(nx, ny, tau_N, tau_R, bc_x, bc_y, de, sides)
    lat.set_populations(f0)
    steps = 6
    lat.step(steps)
    T = um.step_matrix(nx, ny, p["tau"], p["tau_r"], bc_x, bc_y, de, sides)
    v = np.concatenate([f0.ravel(), [1.0]])
    for _ in range(steps):
        v = T @ v
    assert np.isfinite(lat.f).all()
    np.testing.assert_allclose(lat.f.ravel(), v[:-1], atol=1e-13, rtol=0)


def test_diffuse_sides_equal_walls():
    """Two diffuse y sides (Eq. 58 through the per-side pass) reproduce the
    wall rows (Eq. 58 through the wall pass) exactly."""
    rng = np.random.default_rng(3)
    e = 1 + rng.uniform(-1e-3, 1e-3, (6, 7))
    a = oracle.run(7, 6, 0.8, 5.0, e, steps=40, bc_x=oracle.PERIODIC_GRADIENT,
                   bc_y=oracle.WALLS, delta_e=2e-3)
    b = oracle.run(7, 6, 0.8, 5.0, e, steps=40, bc_x=oracle.PERIODIC_GRADIENT, bc_y=S,
                   delta_e=2e-3)
    np.testing.assert_array_equal(a.f, b.f)


def test_side_nodes_satisfy_eqs_55_to_58():
    tau_N, tau_R = 0.7, 1.9
    kap = oracle.kappa(tau_R)
    rng = np.random.default_rng(5)
    e = 1 + rng.uniform(-1e-3, 1e-3, (6, 8))
    # isothermal x sides, diffuse bottom, heat flux q0 into the top
    q0 = 2e-4
    lat = oracle.run(8, 6, tau_N, tau_R, e, steps=23, bc_x=S, bc_y=S,
                     sides=[(ISO, 1.002), (ISO, 0.999), (DIF, 0.0), (FLX, q0)])
    E, qx, qy = lat.moments()
    np.testing.assert_allclose(E[:, 0], 1.002, rtol=1e-15)         # Eq. 55
    np.testing.assert_allclose(E[:, -1], 0.999, rtol=1e-15)
    np.testing.assert_allclose(lat.f[:, 0], np.outer(np.ones(6), oracle.OMEGA) * 1.002,
                               rtol=1e-15)
    np.testing.assert_allclose(qx[:, [0, -1]], 0.0, atol=1e-18)
    np.testing.assert_allclose(qy[0, 1:-1], 0.0, atol=1e-16)       # Eq. 58
    # Eq. 56: q0 = -kappa sum (c.n) e with n = (0, 1), i.e. q_y = -q0
    np.testing.assert_allclose(qy[-1, 1:-1], -q0, rtol=1e-9)
    assert kap < 1
    # flux into the left side of a film, Eq. 57 with n = (-1, 0)
    lat = oracle.run(9, 3, tau_N, tau_R, np.ones((3, 9)), steps=17, bc_x=S,
                     sides=[(FLX, q0), (DIF, 0.0), (DIF, 0.0), (DIF, 0.0)])
    _, qx, _ = lat.moments()
    np.testing.assert_allclose(qx[:, 0], q0, rtol=1e-9)
    np.testing.assert_allclose(qx[:, -1], 0.0, atol=1e-16)


# --- Section 3.1.1: transient film between isothermal sides, Eqs. 61-64 -------
def _film(N, t_star, kn_R=1.29e-3, kn_N=1.29e3):
    d = N - 1
    tau_N, tau_R = oracle.tau_from_kn(kn_N, d), oracle.tau_from_kn(kn_R, d)
    e_h, e_c = 1.001, 1.0
    lat = oracle.run(N, 3, tau_N, tau_R, np.full((3, N), e_c), bc_x=S,
                     sides=[(ISO, e_h), (ISO, e_c), (DIF, 0.0), (DIF, 0.0)])
    steps = int(round(t_star * tau_R))
    lat.step(steps)
    e, qx, _ = lat.moments()
    X = np.arange(N) / d
    theta = (e.mean(0) - e_c) / (e_h - e_c)
    Q = qx.mean(0) * d / ((5.0 / 9.0) * tau_R * (e_h - e_c))    # lambda = v_g^2 tau_R / 3
    th_a, Q_a = analytic.fourier_transient_1d(X, steps / tau_R, kn_R)
    return _l1(theta, th_a), _l1(Q, Q_a)


@pytest.mark.parametrize("t_star,tol_t,tol_q", [(3e4, 0.035, 0.08), (1e5, 0.02, 0.045)])
def test_film_transient_follows_eqs_61_62(t_star, tol_t, tol_q):
    et, eq = _film(101, t_star)
    assert et < tol_t and eq < tol_q


def test_film_first_order_convergence_eqs_63_64():
    """Section 3.1.1 (Fig. 4): the error norms at t* = 1e6 fall about in
    proportion to the grid spacing."""
    Ns = np.array([21, 51, 101])
    errs = np.array([_film(N, 1e6) for N in Ns])
    for k in range(2):
        order = -np.polyfit(np.log(Ns - 1), np.log(errs[:, k]), 1)[0]
        assert 0.8 < order < 1.6
    assert errs[-1, 0] < 5e-3 and errs[-1, 1] < 0.035


# --- Section 3.1.2: square with a heat flux on top, Eqs. 65-67 -----------------
def _square(N):
    L = N - 1
    tau_N, tau_R = oracle.tau_from_kn(2e3, L), oracle.tau_from_kn(2e-3, L)
    q0, e_c = 1e-4, 1.0
    lat = oracle.run(N, N, tau_N, tau_R, np.full((N, N), e_c), bc_x=S, bc_y=S,
                     sides=[(ISO, e_c), (ISO, e_c), (ISO, e_c), (FLX, q0)])
    k = 5.0 / 9.0 * tau_R                    # lattice conductivity v_g^2 tau_R / 3
    lat.step(int(4 * L * L / k))             # four diffusion times: steady
    e, qx, qy = lat.moments()
    Y, X = np.mgrid[0:N, 0:N] / L
    th_a, qx_a, qy_a = analytic.square_steady(X, Y)
    th = (e - e_c) * k / (q0 * L)
    errs = []
    for frac in (0.25, 0.5, 0.75):           # the cross-sections of Fig. 5
        r = int(round(frac * L))
        errs.append([_l1(th[r], th_a[r]), _l1(qx[r] / q0, qx_a[r]), _l1(qy[r] / q0, qy_a[r])])
    return np.array(errs)


def test_square_heat_flux_follows_eqs_65_67():
    threads = oracle.get_threads()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        coarse, fine = _square(21), _square(41)
    finally:
        oracle.set_threads(threads)
    assert fine.max() < 0.16
    assert (coarse / fine).min() > 1.8       # first-order (or better) convergence


# --- Section 3.3: cross-plane film, Eqs. 70-71 ---------------------------------
@pytest.mark.parametrize("kn_R,steps,tol_t,tol_q", [
    (0.01, 65000, 2e-3, 0.01),
    # the paper reports a visible deviation of the flux at large Kn_R from
    # the isothermal treatment (Section 3.3); the profile still matches
    (1.0, 20000, 0.02, 0.15),
    (100.0, 20000, 2e-3, 0.2),
])
def test_cross_plane_follows_eqs_70_71(kn_R, steps, tol_t, tol_q):
    N = 301
    d = N - 1
    tau_N, tau_R = oracle.tau_from_kn(0.01, d), oracle.tau_from_kn(kn_R, d)
    e_h, e_c = 1.001, 1.0
    lat = oracle.run(N, 3, tau_N, tau_R, np.full((3, N), e_c), steps=steps, bc_x=S,
                     sides=[(ISO, e_h), (ISO, e_c), (DIF, 0.0), (DIF, 0.0)])
    e, qx, _ = lat.moments()
    X = np.arange(N) / d
    th_a, Q_a = analytic.cross_plane(X, kn_R)
    theta = (e.mean(0) - e_c) / (e_h - e_c)
    core = (X >= 0.1) & (X <= 0.9)
    assert np.abs(theta - th_a)[core].max() < tol_t
    Q = qx.mean(0)[1:-1] / (VG * (e_h - e_c))
    assert np.ptp(Q) < 1e-3 * abs(Q.mean())                 # steady: uniform flux
    assert Q.mean() == pytest.approx(Q_a, rel=tol_q)


# --- Section 3.4: heat pulse into a plate, Appendix B ---------------------------
def _plate(N, kn_R, kn_N=1.29e-3, q0=1e-4):
    d = N - 1
    tau_N, tau_R = oracle.tau_from_kn(kn_N, d), oracle.tau_from_kn(kn_R, d)
    n_p = int(round(100 * tau_N))            # pulse of 100 tau_N, whole steps
    lat = oracle.run(N, 3, tau_N, tau_R, np.ones((3, N)), bc_x=S,
                     sides=[(FLX, q0), (DIF, 0.0), (DIF, 0.0), (DIF, 0.0)])
    return lat, tau_N, n_p


@pytest.mark.parametrize("kn_R,tol_t,tol_q", [
    (1.29e3, 0.03, 0.03),       # second sound
    (1.29, 0.025, 0.03),        # damped second sound
    (1.29e-3, 3e-3, 0.05),      # diffusive: Q decays, its relative norm grows
])
def test_heat_pulse_follows_appendix_b(kn_R, tol_t, tol_q):
    N = 401
    lat, tau_N, n_p = _plate(N, kn_R)
    q0 = lat.sides[0][1]
    lat.step(n_p)
    _, qx, _ = lat.moments()
    np.testing.assert_allclose(qx[:, 0], q0, rtol=1e-9)       # Eq. 56 during the pulse
    lat.set_side(0, DIF, 0.0)                                   # then adiabatic, Eq. 58
    X = np.arange(N) / (N - 1)
    for t_star in (300.0, 600.0, 1200.0):
        lat.step(int(round(t_star * tau_N)) - lat.step_count)
        e, qx, _ = lat.moments()
        t_eff = lat.step_count / tau_N
        th_a, Q_a = analytic.heat_pulse(X, t_eff, 1.29e-3, kn_R, t_pulse=n_p / tau_N,
                                        gamma_t=9.0)
        assert _l1((e.mean(0) - 1.0) * VG / q0, th_a) < tol_t
        assert _l1(qx.mean(0) / q0, Q_a) < tol_q
        np.testing.assert_allclose(qx[:, 0], 0.0, atol=1e-15)


def test_second_sound_arrival_speed():
    """Section 3.4: in the drift regime the signal crosses the plate at
    v_g / sqrt(3); arrival = the rear side reaching half its first peak."""
    N = 401
    lat, tau_N, n_p = _plate(N, 1.29e3)
    lat.step(n_p)
    lat.set_side(0, DIF, 0.0)
    rear = []
    for _ in range(700):
        lat.step(1)
        rear.append(lat.moments()[0][:, -1].mean() - 1.0)
    rear = np.array(rear)
    first = np.argmax(rear > 0.5 * rear.max())
    # linear interpolation of the half-height crossing, steps since t = 0
    t_a = n_p + first + (0.5 * rear.max() - rear[first - 1]) / (rear[first] - rear[first - 1])
    assert (N - 1) / t_a == pytest.approx(VG / math.sqrt(3.0), rel=0.02)


def test_heat_pulse_terminal_rise():
    """Section 3.4: with both sides adiabatic after the pulse the plate
    settles at Theta = (energy input) / (heat capacity): q_0 n_p / d in
    energy units, n_p v_g / d as Theta, 100 Kn_N = 0.129 for
    t_p = 100 tau_N."""
    N = 51
    lat, tau_N, n_p = _plate(N, 1.29e-3)
    lat.step(n_p)
    lat.set_side(0, DIF, 0.0)
    lat.step(200000)
    theta = (lat.moments()[0] - 1.0) * VG / 1e-4
    assert np.ptp(theta) < 1e-6
    assert theta.mean() == pytest.approx(n_p * VG / (N - 1), rel=1e-4)
    assert theta.mean() == pytest.approx(0.129, rel=2e-3)
