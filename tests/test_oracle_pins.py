"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's formulas: each compares it with a
printed value, a closed form, an invariant, an independent matrix
construction, or a continuum solution from the paper.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import update_matrix as um
from paper_2010_01847_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VG2 = 5.0 / 3.0          # v_g^2 in lattice units (Eq. 48 with c = 1)
CX, CY, W = oracle.CX, oracle.CY, oracle.OMEGA


def _rand_params(rng):
    tau_N = rng.uniform(0.2, 5.0)
    tau_R = rng.uniform(0.6, 80.0)
    return tau_N, tau_R, oracle.params(tau_N, tau_R)


# --- P10: the paper's printed relaxation times (Eqs. 48-49) ---------------
def test_paper_relaxation_times():
    with open(os.path.join(GOLDEN, "paper_relaxation_times.json")) as fh:
        table = json.load(fh)
    for case in table["cases"]:
        d = case["grid_points"] - 1
        tau_N = oracle.tau_from_kn(case["kn_N"], d)
        tau_R = oracle.tau_from_kn(case["kn_R"], d)
        tau = oracle.params(tau_N, tau_R)["tau"]
        assert round(tau, 4) == pytest.approx(case["tau"], abs=1e-12), case


# --- P1: moments of the equilibrium and the source (Eqs. 22-28) ------------
def test_equilibrium_moments_eqs_22_to_25():
    rng = np.random.default_rng(1)
    for _ in range(20):
        e, qx, qy = rng.uniform(-2, 2, 3)
        feq = oracle.equilibrium(e, qx, qy)
        q = np.array([qx, qy])
        c = np.stack([CX, CY], 1).astype(float)
        assert feq.sum() == pytest.approx(e, abs=1e-14)                      # Eq. 22
        np.testing.assert_allclose(c.T @ feq, q, atol=1e-14)                 # Eq. 23
        second = np.einsum("ia,ib,i->ab", c, c, feq)
        np.testing.assert_allclose(second, (5 / 9) * e * np.eye(2), atol=1e-14)  # Eq. 24
        third = np.einsum("ia,ib,ig,i->abg", c, c, c, feq)
        d = np.eye(2)
        expect = (np.einsum("a,bg->abg", q, d) + np.einsum("b,ag->abg", q, d)
                  + np.einsum("g,ab->abg", q, d)) / 3.0
        np.testing.assert_allclose(third, expect, atol=1e-14)               # Eq. 25


def test_source_moments_eqs_26_to_28():
    rng = np.random.default_rng(2)
    c = np.stack([CX, CY], 1).astype(float)
    for _ in range(20):
        qx, qy = rng.uniform(-1, 1, 2)
        tau = rng.uniform(0.55, 5)
        tau_r = rng.uniform(0.6, 100)
        s = oracle.source(qx, qy, tau, tau_r)
        F = -np.array([qx, qy]) / tau_r                      # F = -q / tau_R
        assert s.sum() == pytest.approx(0.0, abs=1e-15)                      # Eq. 26
        np.testing.assert_allclose(c.T @ s, (1 - 1 / (2 * tau)) * F, atol=1e-15)  # Eq. 27
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, s),
                                   np.zeros((2, 2)), atol=1e-15)            # Eq. 28
    assert np.all(oracle.source(0.3, -0.2, 1.3, math.inf) == 0.0)


def test_weights_and_flux_factor():
    # Eqs. 17-18 sum rules used by the Chapman-Enskog expansion
    assert W.sum() == pytest.approx(1.0, abs=1e-15)
    e, qx, qy = oracle.node_moments(oracle.equilibrium(1.0, 0.0, 0.0), 7.0)
    assert (e, qx, qy) == pytest.approx((1.0, 0.0, 0.0), abs=1e-15)
    # Eq. 54 prefactor, and 1 without resistive scattering
    f = np.arange(1.0, 9.0)
    m = float(CX @ f)
    assert oracle.node_moments(f, 3.0)[1] == pytest.approx(m * 6 / 7, rel=1e-15)
    assert oracle.node_moments(f, math.inf)[1] == pytest.approx(m, rel=1e-15)


# --- P2/P3: conservation by the collision ------------------------------------
def test_collision_conserves_energy_and_normal_flux():
    rng = np.random.default_rng(3)
    for _ in range(50):
        tau_N, tau_R, p = _rand_params(rng)
        f = rng.uniform(0, 1, 8)
        post = oracle.collide_node(f, p["tau"], p["tau_r"])
        assert post.sum() == pytest.approx(f.sum(), rel=1e-14)
        # normal scattering only: heat flux conserved
        pn = oracle.params(tau_N, math.inf)
        post_n = oracle.collide_node(f, pn["tau"], math.inf)
        assert CX @ post_n == pytest.approx(CX @ f, abs=1e-14)
        assert CY @ post_n == pytest.approx(CY @ f, abs=1e-14)
        # with resistive scattering the first moment shrinks by
        # (2 tau_r - 1)/(2 tau_r + 1), independent of tau (Eqs. 16, 27, 54)
        ratio = (2 * tau_R - 1) / (2 * tau_R + 1)
        assert CX @ post == pytest.approx(ratio * (CX @ f), abs=1e-14)
        assert CY @ post == pytest.approx(ratio * (CY @ f), abs=1e-14)


def test_uniform_flux_decay_on_lattice():
    tau_N, tau_R = 0.8, 12.0
    n = 37
    lat = oracle.run(6, 5, tau_N, tau_R, 1.0, 0.01, -0.004)
    # Eq. 15 puts sum c_i e_i = q; Eq. 54 then reports kappa q at step 0
    kap = 2 * tau_R / (2 * tau_R + 1)
    _, qx0, qy0 = lat.moments()
    np.testing.assert_allclose(qx0, 0.01 * kap, rtol=1e-13)
    lat.step(n)
    e, qx, qy = lat.moments()
    ratio = ((2 * tau_R - 1) / (2 * tau_R + 1)) ** n
    np.testing.assert_allclose(e, 1.0, atol=1e-14)
    np.testing.assert_allclose(qx, 0.01 * kap * ratio, rtol=1e-12)
    np.testing.assert_allclose(qy, -0.004 * kap * ratio, rtol=1e-12)


# --- P4/P12: exact Fourier-mode evolution on a periodic lattice -------------
@pytest.mark.parametrize("mx,my", [(1, 0), (0, 1), (1, 1), (3, 2)])
def test_fourier_mode_exact(mx, my):
    nx, ny = 24, 16
    tau_N, tau_R = 0.9, 7.5
    p = oracle.params(tau_N, tau_R)
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    y, x = np.mgrid[0:ny, 0:nx]
    ph = kx * x + ky * y
    A, Bq = 1e-3, 4e-4
    e = 1.0 + A * np.cos(ph)
    qx = Bq * np.cos(ph)               # a travelling component
    lat = oracle.run(nx, ny, tau_N, tau_R, e, qx, 0 * qx)
    steps = 23
    lat.step(steps)
    # exact: complex amplitudes F_i with f_i - w_i = Re(F_i exp(i k.x))
    F0 = oracle.equilibrium(A, Bq, 0.0).astype(complex)
    Mk = um.mode_matrix(kx, ky, p["tau"], p["tau_r"])
    Fn = np.linalg.matrix_power(Mk, steps) @ F0
    expect = W[None, None, :] + np.real(Fn[None, None, :] * np.exp(1j * ph)[..., None])
    np.testing.assert_allclose(lat.f, expect, atol=1e-14, rtol=0)


def test_isotropy_x_vs_y():
    # the same mode along x and along y decays identically (lattice symmetry)
    n = 32
    tau_N, tau_R = 1.7, 20.0
    ex = inputs.sine_mode(n, 4, 16.0, 1e-3, direction="x")
    ey = inputs.sine_mode(4, n, 16.0, 1e-3, direction="y")
    lx = oracle.run(n, 4, tau_N, tau_R, ex, steps=40)
    ly = oracle.run(4, n, tau_N, tau_R, ey, steps=40)
    np.testing.assert_allclose(lx.moments()[0][0, :], ly.moments()[0][:, 0],
                               atol=1e-15)
    np.testing.assert_allclose(lx.moments()[1][0, :], ly.moments()[2][:, 0],
                               atol=1e-15)


# --- P5: continuum dispersion, Eq. 52 ---------------------------------------
def _eq52_roots(tau_C, tau_R, k):
    b = (0 if math.isinf(tau_R) else 1 / tau_R) + (4 / 15) * tau_C * VG2 * k * k
    c = VG2 * k * k / 3
    return np.roots([1.0, b, c])


def test_fourier_limit_decay_rate():
    """Resistive scattering only: the slow root of Eq. 52 ~ -(5/9) tau_R k^2."""
    nx, tau_R = 256, 2.0
    k = 2 * np.pi / nx
    x = np.arange(nx)
    lat = oracle.run(nx, 2, math.inf, tau_R, 1 + 1e-3 * np.cos(k * x)[None, :].repeat(2, 0))
    amp = lambda: 2 * np.mean((lat.moments()[0] - 1) * np.cos(k * x)[None, :])
    lat.step(200)
    a1 = amp()
    lat.step(1000)
    s = math.log(amp() / a1) / 1000
    s_slow = max(_eq52_roots(oracle.params(math.inf, tau_R)["tau_C"], tau_R, k).real)
    assert s == pytest.approx(s_slow, rel=1e-4)
    assert s == pytest.approx(-(5 / 9) * tau_R * k * k, rel=2e-3)   # Fourier's law


def test_damped_mode_follows_eq52():
    """Sine mode with the 8192^2 heat-mode workload's relaxation times:
    T(t)/T(0) = (s2 e^{s1 t} - s1 e^{s2 t})/(s2 - s1) with q(0) = 0."""
    w = inputs.THROUGHPUT_8192
    tau_N = oracle.tau_from_kn(w.kn_N, w.length)
    tau_R = oracle.tau_from_kn(w.kn_R, w.length)
    p = oracle.params(tau_N, tau_R)
    k = 2 * np.pi / 512
    s1, s2 = _eq52_roots(p["tau_C"], tau_R, k)
    x = np.arange(512)
    lat = oracle.run(512, 2, tau_N, tau_R, inputs.sine_mode(512, 2, 512.0, 1e-3))
    for n in (100, 300, 600, 1000):
        lat.step(n - lat.step_count)
        amp = 2 * np.mean((lat.moments()[0] - 1) * np.sin(k * x)[None, :]) / 1e-3
        th = (s2 * np.exp(s1 * n) - s1 * np.exp(s2 * n)) / (s2 - s1)
        assert amp == pytest.approx(th, rel=1e-3), n


# --- P6: second-sound speed v_g / sqrt(3) (Section 3.4) ----------------------
@pytest.mark.parametrize("kn_R", [10.0, 1.0])
def test_second_sound_speed(kn_R):
    with open(os.path.join(GOLDEN, "second_sound_speed.json")) as fh:
        speed = json.load(fh)["speed_cells_per_step"]
    w = inputs.second_sound_4096x4(kn_R)
    lat = oracle.run(w.nx, w.ny, oracle.tau_from_kn(w.kn_N, w.length),
                     oracle.tau_from_kn(w.kn_R, w.length),
                     *inputs.initial_fields(w))
    pos = []
    for n in (1000, 2000):
        lat.step(n - lat.step_count)
        prof = lat.moments()[0].mean(0)[w.nx // 2:]
        j = int(np.argmax(prof))
        y0, y1, y2 = prof[j - 1:j + 2]
        pos.append(j + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2))
    assert (pos[1] - pos[0]) / 1000 == pytest.approx(speed, rel=1e-3)


# --- P7/P8/P9: phonon Poiseuille flow, Eqs. 68-69, periodic gradient --------
def eq68(Y, kn_N, kn_R):
    kn_C = 1 / (1 / kn_N + 1 / kn_R)
    ke = math.sqrt(kn_C * kn_R / 5)
    den = 1 + math.exp(-1 / ke) + 8 / 15 * kn_C / ke * (1 - math.exp(-1 / ke))
    return 1 - (np.exp((Y - 1) / ke) + np.exp(-Y / ke)) / den


def eq69(kn_N, kn_R):
    kn_C = 1 / (1 / kn_N + 1 / kn_R)
    ke = math.sqrt(kn_C * kn_R / 5)
    den = 1 + math.exp(-1 / ke) + 8 / 15 * kn_C / ke * (1 - math.exp(-1 / ke))
    return 1 - 2 * ke * (1 - math.exp(-1 / ke)) / den


def _channel(nx, ny, kn_N, kn_R, steps, delta_e=1e-3):
    d = ny - 1
    tau_N, tau_R = oracle.tau_from_kn(kn_N, d), oracle.tau_from_kn(kn_R, d)
    lat = oracle.run(nx, ny, tau_N, tau_R, np.ones((ny, nx)), steps=steps,
                     bc_x=oracle.PERIODIC_GRADIENT, bc_y=oracle.WALLS,
                     delta_e=delta_e)
    return lat, oracle.params(tau_N, tau_R)


@pytest.mark.parametrize("nx,ny,kn_R,steps,core_tol,mean_tol", [
    (3, 301, 1.0, 20000, 2e-3, 0.01),       # Section 3.2 grid
    (3, 301, 100.0, 150000, 1e-2, 0.02),    # Section 3.2 grid, Poiseuille
    (128, 32, 1.0, 10000, 5e-3, 0.01),      # 128x32 channel
])
def test_poiseuille_eq68_eq69(nx, ny, kn_R, steps, core_tol, mean_tol):
    lat, p = _channel(nx, ny, 0.01, kn_R, steps)
    e, qx, qy = lat.moments()
    slope = np.polyfit(np.arange(nx), e.mean(0), 1)[0]
    Q = qx.mean(1) / (-(5 / 9) * p["tau_r"] * slope)
    Y = np.arange(ny) / (ny - 1)
    core = (Y >= 0.2) & (Y <= 0.8)
    assert np.abs(Q - eq68(Y, 0.01, kn_R))[core].max() < core_tol
    assert Q.mean() == pytest.approx(eq69(0.01, kn_R), rel=mean_tol)
    assert np.abs(qy).max() < 1e-9 * np.abs(qx).max()  # round-off of e ~ 1


def test_periodic_gradient_steady_state_is_affine():
    nx, ny, de = 16, 12, 2e-3
    lat, p = _channel(nx, ny, 0.05, 0.5, 6000, de)
    e, qx, _ = lat.moments()
    # e(x+1) - e(x) = -delta_e / nx everywhere, q independent of x
    np.testing.assert_allclose(np.diff(e, axis=1), -de / nx, rtol=1e-8, atol=0)
    np.testing.assert_allclose(qx, qx[:, :1].repeat(nx, 1), atol=1e-15)
    assert qx.min() > 0             # hot on the left (Eq. 59) drives +x flux


# --- P13: brute force against the explicit update matrix --------------------
@pytest.mark.parametrize("nx,ny,bc_x,bc_y,de", [
    (4, 3, oracle.PERIODIC_GRADIENT, oracle.WALLS, 0.37),
    (5, 4, oracle.PERIODIC_GRADIENT, oracle.PERIODIC, -0.21),
    (3, 5, oracle.PERIODIC, oracle.WALLS, 0.0),
    (3, 3, oracle.PERIODIC, oracle.PERIODIC, 0.0),
])
def test_brute_force_matrix(nx, ny, bc_x, bc_y, de):
    tau_N, tau_R = 0.7, 3.3
    p = oracle.params(tau_N, tau_R)
    rng = np.random.default_rng(7)
    f0 = rng.uniform(0.0, 0.3, (ny, nx, 8))
    lat = oracle.Lattice(nx, ny, tau_N, tau_R, bc_x, bc_y, de)
    lat.set_populations(f0)
    steps = 7
    lat.step(steps)
    T = um.step_matrix(nx, ny, p["tau"], p["tau_r"], bc_x, bc_y, de)
    v = np.concatenate([f0.ravel(), [1.0]])
    for _ in range(steps):
        v = T @ v
    np.testing.assert_allclose(lat.f.ravel(), v[:-1], atol=1e-13, rtol=0)


def test_wall_nodes_have_zero_normal_flux():
    lat, _ = _channel(8, 9, 0.02, 2.0, 57)
    f = lat.f
    for y in (0, lat.ny - 1):
        np.testing.assert_allclose(f[y] @ CY, 0.0, atol=1e-16)


def test_energy_conserved_periodic_with_seam():
    e, qx, qy = inputs.random_state_fields(10, 7, seed=5)
    lat = oracle.run(10, 7, 0.6, 9.0, e, qx, qy, bc_x=oracle.PERIODIC_GRADIENT,
                     delta_e=0.05)
    total0 = lat.f.sum()
    lat.step(100)
    assert lat.f.sum() == pytest.approx(total0, rel=1e-13)


def test_thread_count_does_not_change_results():
    e, qx, qy = inputs.random_state_fields(33, 20, seed=9)
    runs = []
    for t in (1, 3):
        oracle.set_threads(t)
        lat = oracle.run(33, 20, 0.7, 5.0, e, qx, qy, steps=15,
                         bc_x=oracle.PERIODIC_GRADIENT, bc_y=oracle.WALLS,
                         delta_e=0.01)
        runs.append(lat.f.copy())
    oracle.set_threads(1)
    assert np.array_equal(runs[0], runs[1])


# --- linear stability of the scheme near tau -> 1/2 ---------------------------
def test_instability_below_tau_bound_matches_mode_matrix():
    """The D2Q8 scheme without a rest population is linearly unstable for
    tau below ~0.576 (tau_r = inf): the exact mode matrix has spectral radius
    > 1 near k = (2.06, pi).  The looped oracle must grow at exactly the rate
    the matrix predicts (64 x 2 lattice: k = 2 pi 21/64 and pi are on it), and
    stay bounded just above the bound."""
    nx, ny = 64, 2
    kx, ky = 2 * np.pi * 21 / nx, np.pi
    for tau, grows in ((0.55, True), (0.6, False)):
        tau_N = tau - 0.5
        Mk = um.mode_matrix(kx, ky, tau, math.inf)
        rho = np.abs(np.linalg.eigvals(Mk)).max()
        assert (rho > 1 + 1e-6) == grows
        e = 1 + 1e-6 * inputs.uniform_noise((ny, nx), 1.0, seed=3)
        lat = oracle.run(nx, ny, tau_N, math.inf, e)
        lat.step(400)
        a = np.linalg.norm(lat.f - oracle.OMEGA)
        lat.step(200)
        b = np.linalg.norm(lat.f - oracle.OMEGA)
        if grows:
            # the largest growing mode on this lattice dominates after 400
            # steps; its complex eigenvalue makes the norm oscillate slightly
            rates = [np.abs(np.linalg.eigvals(um.mode_matrix(2 * np.pi * m / nx, np.pi * j, tau,
                                                               math.inf))).max()
                     for m in range(nx) for j in (0, 1)]
            assert (b / a) ** (1 / 200) == pytest.approx(max(rates), rel=1e-4)
        else:
            assert b <= 1e-5


# --- warm-start network reference ---------------------------------------------
def test_mlp_gelu_identities():
    from oracle import mlp
    x = np.linspace(-6, 6, 101)
    g = mlp.gelu(x)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu(-x), g - x, atol=1e-15)      # Phi(-x) = 1 - Phi(x)
    np.testing.assert_allclose(mlp.gelu(np.array([8.0]))[0], 8.0, rtol=1e-14)
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h),
                               atol=1e-8)


def test_mlp_gradient_against_central_differences():
    from oracle import mlp
    widths = [3, 7, 5, 4]
    rng = np.random.default_rng(4)
    n = sum(a * b + b for a, b in zip(widths[:-1], widths[1:]))
    p = rng.normal(0, 0.7, n)
    x = rng.normal(0, 1, (6, 3))
    t = rng.normal(0, 1, (6, 4))
    loss, g = mlp.loss_grad(p, widths, x, t)
    h = 1e-6
    num = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        num[i] = (mlp.loss_grad(p + e, widths, x, t)[0] - mlp.loss_grad(p - e, widths, x, t)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)
    # a network with no hidden layer is a least-squares fit: gradient closed form
    W = rng.normal(size=(2, 3))
    b = rng.normal(size=2)
    t2 = rng.normal(size=(6, 2))
    l2, g2 = mlp.loss_grad(np.concatenate([W.ravel(), b]), [3, 2], x, t2)
    r = x @ W.T + b - t2
    np.testing.assert_allclose(g2[:6], (2 * r.T @ x / r.size).ravel(), rtol=1e-13)
    np.testing.assert_allclose(g2[6:], 2 * r.sum(0) / r.size, rtol=1e-13)
