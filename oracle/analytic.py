"""Continuum solutions the paper compares its boundary treatments with.

TEST INFRASTRUCTURE (part of the oracle): only the tests import this module.
Each function evaluates a closed form printed in Section 3 or Appendix B of
Guo & Wang (arXiv 2010.01847) in the paper's non-dimensional variables.
They are references for the lattice results of the oracle, which tends to
them as the grid is refined (first order, Eqs. 63-64), not equal to them.

  fourier_transient_1d   Eqs. 61-62   film between two isothermal sides
  square_steady          Eqs. 65-67   square, heat flux on top, three
                                       isothermal sides
  cross_plane            Eqs. 70-71   film, hydrodynamic model with the
                                       temperature-jump condition
  heat_pulse             Eqs. B9-B13  plate heated by a flux pulse, Laplace
                                       domain, inverted by Eq. B16
"""
from __future__ import annotations

import math

import numpy as np


def fourier_transient_1d(X, t_star, kn_R, terms=4000):
    """Eqs. 61-62: Theta = (T - T_c)/(T_h - T_c) and
    Q = q_x d / (lambda (T_h - T_c)) at X = x/d and t* = t/tau_R, for a film
    at T_c whose side X = 0 is raised to T_h at t* = 0."""
    X = np.asarray(X, dtype=np.float64)
    n = np.arange(1, terms + 1, dtype=np.float64)[:, None]
    decay = np.exp(-(kn_R ** 2) * n ** 2 * math.pi ** 2 * t_star / 3.0)
    theta = 1.0 - X - (2.0 / math.pi) * (np.sin(n * math.pi * X) / n * decay).sum(0)
    Q = 1.0 + 2.0 * (np.cos(n * math.pi * X) * decay).sum(0)
    return theta, Q


def square_steady(X, Y, Q0=1.0, terms=400):
    """Eqs. 65-67: steady Theta, Q_x, Q_y in the unit square with Theta = 0
    on X = 0, X = 1 and Y = 0 and the incident flux Q0 on Y = 1.
    sinh(n pi Y)/cosh(n pi) and cosh(n pi Y)/cosh(n pi) are evaluated as
    exp(n pi (Y - 1)) (1 -+ exp(-2 n pi Y)) / (1 + exp(-2 n pi)) so large n
    does not overflow."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = np.arange(1, terms + 1, dtype=np.float64).reshape((-1,) + (1,) * X.ndim)
    npi = n * math.pi
    odd = 1.0 - np.cos(npi)                   # 1 - cos(n pi): 2 for odd n, 0 for even
    base = np.exp(npi * (Y - 1.0)) / (1.0 + np.exp(-2.0 * npi))
    sh = base * (1.0 - np.exp(-2.0 * npi * Y))
    ch = base * (1.0 + np.exp(-2.0 * npi * Y))
    theta = (2.0 * Q0 / npi ** 2 * odd * np.sin(npi * X) * sh).sum(0)
    Qx = -(2.0 * Q0 / npi * odd * np.cos(npi * X) * sh).sum(0)
    Qy = -(2.0 * Q0 / npi * odd * np.sin(npi * X) * ch).sum(0)
    return theta, Qx, Qy


def cross_plane(X, kn_R):
    """Eqs. 70-71: Theta = (T - T_c)/(T_h - T_c) and
    Q = q_x / (C_V v_g (T_h - T_c)) across a film between isothermal
    sides."""
    X = np.asarray(X, dtype=np.float64)
    den = 1.0 + 4.0 * kn_R / 3.0
    theta = -X / den + (1.0 + 2.0 * kn_R / 3.0) / den
    return theta, (kn_R / 3.0) / den


def laplace_inverse(F, t, gamma_t=3.0, terms=2000):
    """Eq. B16 with T_p = t (Eqs. B14-B15): f(t) ~ exp(gamma t)/t
    [F(gamma)/2 + Re sum_n F(gamma + i n pi / t) (-1)^n].  ``F`` maps an
    array of complex s (last axis) to transforms of the same shape (leading
    axes free).  The alternating sum is cut after ``terms`` terms and the
    last two partial sums are averaged.  gamma t = 3 is the paper's choice;
    the discretisation error is of order exp(-2 gamma t) relative."""
    gamma = gamma_t / t
    n = np.arange(0, terms + 1, dtype=np.float64)
    s = gamma + 1j * n * math.pi / t
    sign = np.where(n == 0, 0.5, np.where(n % 2 == 0, 1.0, -1.0))
    terms_re = (F(s) * sign).real
    partial = np.cumsum(terms_re, axis=-1)
    return math.exp(gamma_t) / t * 0.5 * (partial[..., -1] + partial[..., -2])


def heat_pulse_transforms(X, kn_N, kn_R, t_pulse=100.0):
    """Eqs. B9-B13: returns F(s) -> (Theta_bar, Q_bar) at the points X for
    the plate of Section 3.4 heated at X = 0 by Q = 1 during
    0 < t* < t_pulse (t* = t/tau_N), adiabatic at X = 1.  The term
    C_1 exp(A X) = -C_2 exp(-A (2 - X)) (Eq. B12) is formed that way so
    large |A| does not overflow."""
    kn_C = 1.0 / (1.0 / kn_N + 1.0 / kn_R)
    X = np.asarray(X, dtype=np.float64)[:, None]

    def both(s):
        s = np.asarray(s, dtype=np.complex128)[None, :]
        A = np.sqrt((kn_R / kn_N * s + 1.0) /
                    (kn_N * kn_R / (3.0 * s) + 4.0 / 15.0 * kn_C * kn_R))
        A = np.where(A.real < 0, -A, A)              # the root that decays
        C2 = (1.0 / s) * (1.0 - np.exp(-t_pulse * s)) / (1.0 - np.exp(-2.0 * A))
        up = -C2 * np.exp(-A * (2.0 - X))            # C_1 exp(A X)
        down = C2 * np.exp(-A * X)                   # C_2 exp(-A X)
        Qb = up + down                               # Eq. B10
        Tb = -(kn_N / s) * (A * up - A * down)       # Eq. B13
        return Tb, Qb

    return both


def heat_pulse(X, t_star, kn_N, kn_R, t_pulse=100.0, gamma_t=3.0, terms=2000):
    """Theta = (T - T_0) C_V v_g / q_0 and Q = q_x / q_0 (Eq. 76) at X and
    t* = t / tau_N for the heat pulse of Section 3.4 (Appendix B)."""
    both = heat_pulse_transforms(X, kn_N, kn_R, t_pulse)
    theta = laplace_inverse(lambda s: both(s)[0], t_star, gamma_t, terms)
    Q = laplace_inverse(lambda s: both(s)[1], t_star, gamma_t, terms)
    return theta, Q
