"""The collision as the FP32 kernels arrange it, in FP64 against the oracle.

The kernels relax towards w_i rho + h_i c_i.(1 - zeta) m with the single rate
omega = 1/tau, zeta = lambda + sigma tau (1 - lambda), which folds the
resistive source of Eq. 16 into the relaxation of Eq. 13.  In exact
arithmetic that is the same update as Eq. 13 with Eqs. 15-16 and 54; these
checks hold the identity (and the coefficients it uses) against the
oracle's own collision on random populations, so a wrong fold (a sign, a
missing (1 - lambda), tau in place of tau_r) fails here on the CPU."""
import math

import numpy as np
import pytest

import oracle

# directions of Eq. 14 in the kernels' order (index i = the paper's i + 1)
CX = np.array([1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
W = np.array([2 / 9] * 4 + [1 / 36] * 4)
H = np.array([1 / 3] * 4 + [1 / 12] * 4)


def folded(f, tau, tau_r):
    """d* = d - omega (d - w rho - h c.(1 - zeta) m)."""
    omega = 1.0 / tau
    resistive = math.isfinite(tau_r)
    lam = 1.0 / (2.0 * tau_r + 1.0) if resistive else 0.0
    sigma = (1.0 - 1.0 / (2.0 * tau)) / tau_r if resistive else 0.0
    zeta = lam + sigma * tau * (1.0 - lam)
    rho = f.sum()
    mx, my = (CX * f).sum(), (CY * f).sum()
    t = H * (CX * mx + CY * my) * (1.0 - zeta)
    return f - omega * (f - W * rho - t)


def separate(f, tau, tau_r):
    """d* = d - omega (d - w rho - t) - sigma t, t = h c.(m - lambda m)."""
    omega = 1.0 / tau
    resistive = math.isfinite(tau_r)
    lam = 1.0 / (2.0 * tau_r + 1.0) if resistive else 0.0
    sigma = (1.0 - 1.0 / (2.0 * tau)) / tau_r if resistive else 0.0
    rho = f.sum()
    mx, my = (CX * f).sum(), (CY * f).sum()
    t = H * (CX * (mx - lam * mx) + CY * (my - lam * my))
    return f - omega * (f - W * rho - t) - sigma * t


@pytest.mark.parametrize("kn_N,kn_R,length", [
    (0.01, 0.1, 512.0),          # the 8192^2 heat mode
    (1e-3, 0.1, 4096.0),         # second sound
    (1e-3, 10.0, 4096.0),
    (0.1, 1.0, 32.0),
    (0.05, math.inf, 64.0),      # no resistive scattering: zeta = 0
])
def test_folded_relaxation_is_the_oracle_collision(kn_N, kn_R, length):
    tau_N = oracle.tau_from_kn(kn_N, length)
    tau_R = oracle.tau_from_kn(kn_R, length) if math.isfinite(kn_R) else math.inf
    p = oracle.params(tau_N, tau_R)
    tau, tau_r = p["tau"], p["tau_r"]
    rng = np.random.default_rng(11)
    for _ in range(20):
        f = W * (1.0 + rng.uniform(-0.1, 0.1)) + rng.normal(0.0, 1e-2, 8)
        want = oracle.collide_node(f, tau, tau_r)
        scale = np.abs(want).max()
        np.testing.assert_allclose(separate(f, tau, tau_r), want, rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(folded(f, tau, tau_r), want, rtol=0, atol=1e-14 * scale)


def test_folded_flux_factor_matches_eq16_decay():
    """The flux after one collision of a uniform state is (1 - omega zeta) m:
    for the second-sound case the fold gives the rate (2 tau_r - 1) /
    (2 tau_r + 1) of the oracle's uniform-flux decay only with zeta as
    defined (a plausible slip, zeta = lambda + sigma tau, misses it)."""
    tau_N = oracle.tau_from_kn(1e-3, 4096.0)
    tau_R = oracle.tau_from_kn(0.1, 4096.0)
    p = oracle.params(tau_N, tau_R)
    tau, tau_r = p["tau"], p["tau_r"]
    f = oracle.equilibrium(1.0, 1e-3, 0.0)
    out = folded(f, tau, tau_r)
    ref = oracle.collide_node(f, tau, tau_r)
    m_out, m_ref = (CX * out).sum(), (CX * ref).sum()
    assert m_out == pytest.approx(m_ref, rel=1e-13)
    lam = 1.0 / (2.0 * tau_r + 1.0)
    sigma = (1.0 - 1.0 / (2.0 * tau)) / tau_r
    wrong_zeta = lam + sigma * tau
    m_in = (CX * f).sum()
    m_wrong = m_in * (1.0 - wrong_zeta / tau)
    assert abs(m_wrong - m_ref) > 1e-6 * abs(m_ref)
