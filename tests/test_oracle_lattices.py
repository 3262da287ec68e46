"""Pins of the D1Q2 / D3Q14 oracle (``oracle/lattices.py``) against what the
paper fixes: the moment conditions of Section 2.3 (Eqs. 22-28), the
conservation properties of the collision, exact Fourier-mode evolution, and
the continuum dispersion of Eqs. 6-7 (Eq. 52 for longitudinal modes, the
nonlocal term of Eq. 7 for transverse ones) and the second-sound speed
v_g / sqrt(3) of Section 3.4.  CPU only."""
import math

import numpy as np
import pytest

from oracle import lattices as lt

D3, D1 = lt.D3Q14, lt.D1Q2


def _rand_state(L, rng, shape=()):
    e = 1 + rng.uniform(-0.1, 0.1, shape)
    q = rng.uniform(-0.05, 0.05, (L.dim,) + shape)
    return e, q


# --- Eqs. 22-28 on the new velocity sets -------------------------------------
@pytest.mark.parametrize("L", [D3, D1], ids=lambda L: L.name)
def test_equilibrium_and_source_moments(L):
    rng = np.random.default_rng(1)
    c = L.c.astype(float)
    I = np.eye(L.dim)
    for _ in range(5):
        e, q = _rand_state(L, rng)
        eq = lt.equilibrium(L, e, q)
        assert eq.sum() == pytest.approx(e, abs=1e-14)                     # Eq. 22
        np.testing.assert_allclose(c.T @ eq, q, atol=1e-15)                 # Eq. 23
        second = np.einsum("ia,ib,i->ab", c, c, eq)
        # Eq. 24: (5/9) c^2 e on D3Q14; c^2 e on D1Q2 (the lattice's own K2)
        K2 = 5 / 9 if L is D3 else 1.0
        np.testing.assert_allclose(second, K2 * e * I, atol=1e-14)
        third = np.einsum("ia,ib,ig,i->abg", c, c, c, eq)
        K4 = 1 / 3 if L is D3 else 1.0
        expect = K4 * (np.einsum("a,bg->abg", q, I) + np.einsum("b,ag->abg", q, I)
                       + np.einsum("g,ab->abg", q, I)) / (3 if L is D1 else 1)
        np.testing.assert_allclose(third, expect, atol=1e-15)              # Eq. 25
    # the collision: energy kept (Eq. 26 with Eq. 22), flux scaled by
    # (2 tau_r - 1)/(2 tau_r + 1) (Eqs. 16, 27, 54), kept for tau_R = inf
    f = rng.uniform(0, 0.2, L.Q)
    for tau_N, tau_R in ((0.8, 6.0), (1.3, math.inf)):
        tau, tau_r = lt.relaxation(tau_N, tau_R)
        post = lt.collide(L, f, tau, tau_r)
        assert post.sum() == pytest.approx(f.sum(), abs=1e-15)
        ratio = 1.0 if math.isinf(tau_r) else (2 * tau_r - 1) / (2 * tau_r + 1)
        np.testing.assert_allclose(c.T @ post, ratio * (c.T @ f), atol=1e-15)


def test_d3q14_weights_are_the_unique_solution():
    """The four conditions of Section 2.3 on 6 axis + 8 corner velocities:
    a 2x2 linear system for each weight class."""
    # w: 6 wa + 8 wc = 1, 2 wa + 8 wc = 5/9; h: 2 ha + 8 hc = 1, 8 hc = 1/3
    wa, wc = np.linalg.solve([[6, 8], [2, 8]], [1, 5 / 9])
    ha, hc = np.linalg.solve([[2, 8], [0, 8]], [1, 1 / 3])
    np.testing.assert_allclose(D3.w, [wa] * 6 + [wc] * 8, rtol=1e-15)
    np.testing.assert_allclose(D3.h, [ha] * 6 + [hc] * 8, rtol=1e-15)


# --- exact evolution of a Fourier mode (brute force) ---------------------------
@pytest.mark.parametrize("L,shape,m", [(D3, (6, 5, 8), (1, 2, 1)), (D3, (4, 4, 4), (0, 0, 1)),
                                       (D1, (16,), (3,))], ids=["d3a", "d3b", "d1"])
def test_fourier_mode_exact(L, shape, m):
    tau_N, tau_R = 0.9, 5.5
    tau, tau_r = lt.relaxation(tau_N, tau_R)
    # k in (x, y, z) order; shape is (nz, ny, nx)
    n_xyz = shape[::-1]
    k = np.array([2 * np.pi * mi / ni for mi, ni in zip(m, n_xyz)])
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")[::-1]   # x, y, z
    ph = sum(ki * g for ki, g in zip(k, grids))
    A, B = 1e-3, 3e-4
    run = lt.Run(L, shape, tau_N, tau_R)
    q = np.zeros((L.dim,) + shape)
    q[0] = B * np.cos(ph)
    run.init(1 + A * np.cos(ph), q)
    steps = 17
    run.step(steps)
    F0 = lt.equilibrium(L, A, np.array([B] + [0.0] * (L.dim - 1))).astype(complex)
    Fn = np.linalg.matrix_power(lt.mode_matrix(L, k, tau, tau_r), steps) @ F0
    expect = L.w.reshape((L.Q,) + (1,) * L.dim) + np.real(
        Fn.reshape((L.Q,) + (1,) * L.dim) * np.exp(1j * ph)[None])
    np.testing.assert_allclose(run.f, expect, atol=1e-14, rtol=0)


# --- continuum limit: Eqs. 6-7 / Eq. 52 -----------------------------------------
def _rates(L, k_vec, tau_N, tau_R):
    tau, tau_r = lt.relaxation(tau_N, tau_R)
    lam = np.linalg.eigvals(lt.mode_matrix(L, k_vec, tau, tau_r))
    return np.log(lam.astype(complex))


def _slowest(s, count):
    return s[np.argsort(-s.real)][:count]


@pytest.mark.parametrize("direction", [(1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 1, 0)])
def test_d3q14_longitudinal_modes_follow_eq52(direction):
    vg2 = 1 / D3.speed ** 2                       # v_g^2 in lattice units (c = 1): 5/3
    tau_N, tau_R = 2.0, 40.0
    tau, tau_r = lt.relaxation(tau_N, tau_R)
    tau_C = tau - 0.5
    for kmag in (2 * np.pi / 128, 2 * np.pi / 256):
        k = kmag * np.asarray(direction, float) / np.linalg.norm(direction)
        # Eq. 52: s^2 + s (1/tau_R + (4/15) tau_C v_g^2 k^2) + (1/3) v_g^2 k^2 = 0
        roots = np.roots([1, 1 / tau_R + 4 / 15 * tau_C * vg2 * kmag ** 2, vg2 * kmag ** 2 / 3])
        s = _slowest(_rates(D3, k, tau_N, tau_R), 5)
        for r in roots:
            best = s[np.argmin(np.abs(s - r))]
            assert abs(best - r) < 3e-3 * abs(r), (direction, kmag, r, best)


@pytest.mark.parametrize("direction", [(1, 0, 0), (1, 1, 1)])
def test_d3q14_transverse_modes_follow_nonlocal_term_of_eq7(direction):
    """q perpendicular to k with uniform T and normal scattering only:
    dq/dt = (1/5) tau_C v_g^2 lap q (Eq. 7 divided by tau_R), a decay
    rate of (1/5) tau_C v_g^2 k^2."""
    vg2 = 1 / D3.speed ** 2
    tau_N, tau_R = 3.0, math.inf          # normal scattering only: the flux is not damped
    tau, tau_r = lt.relaxation(tau_N, tau_R)
    tau_C = tau - 0.5
    d = np.asarray(direction, float) / np.linalg.norm(direction)
    s0 = 0.0                              # uniform flux (k = 0) is conserved
    errs = []
    for kmag in (2 * np.pi / 256, 2 * np.pi / 512):
        s = _rates(D3, kmag * d, tau_N, tau_R)
        # the two transverse modes: real rates closest to s0, degenerate
        cand = np.sort(s.real[np.abs(s.imag) < 1e-9])[::-1]
        cand = cand[np.argsort(np.abs(cand - s0))][:2]
        extra = -0.2 * tau_C * vg2 * kmag ** 2
        errs.append(np.abs((cand - s0) - extra).max() / abs(extra))
    # the lattice adds O(k^2) to the coefficient: small, and shrinking as k^2
    assert errs[0] < 5e-3 and errs[1] < errs[0] / 3.5


def test_d3q14_second_sound_speed():
    """Normal scattering only, small tau_N: the wave speed is v_g / sqrt(3)
    (Section 3.4) = sqrt(5)/3 cells per step, the same along every axis."""
    for direction in ((1, 0, 0), (1, 1, 0), (1, 1, 1)):
        d = np.asarray(direction, float) / np.linalg.norm(direction)
        kmag = 2 * np.pi / 400
        s = _rates(D3, kmag * d, 0.3, math.inf)
        osc = s[np.abs(s.imag) > 1e-6]
        wave = osc[np.argmax(osc.real)]
        assert abs(wave.imag) / kmag == pytest.approx(math.sqrt(5) / 3, rel=1e-3)


def test_d1q2_follows_the_cattaneo_equation():
    """D1Q2 recovers Eqs. 6-7 without the nonlocal term: s^2 + s / tau_R +
    (1/3) v_g^2 k^2 = 0 with v_g = sqrt(3) c, i.e. s^2 + s/tau_R + k^2 = 0."""
    tau_N, tau_R = 1.5, 30.0
    for kmag in (2 * np.pi / 200, 2 * np.pi / 400):
        s = _rates(D1, np.array([kmag]), tau_N, tau_R)
        roots = np.roots([1, 1 / tau_R, kmag ** 2])
        for r in roots:
            assert np.min(np.abs(s - r)) < 2e-3 * abs(r)


def test_runs_conserve_energy():
    rng = np.random.default_rng(9)
    for L, shape in ((D3, (5, 6, 7)), (D1, (33,))):
        run = lt.Run(L, shape, 0.7, 3.0)
        e, q = _rand_state(L, rng, shape)
        run.init(e, q)
        E0 = run.f.sum()
        run.step(25)
        assert run.f.sum() == pytest.approx(E0, rel=1e-14)
