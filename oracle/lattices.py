"""FP64 reference of the phonon lattice Boltzmann scheme on the D1Q2 and
D3Q14 lattices (Guo & Wang, arXiv 2010.01847).

TEST INFRASTRUCTURE (part of the oracle): only the tests import this module;
it shares nothing with the CUDA path.

Section 2.2 states that the scheme extends to the one-dimensional D1Q2 and
three-dimensional D3Q14 lattices but gives no weights for them.  The weights
here come from the moment conditions the Chapman-Enskog analysis of
Section 2.3 rests on, written for the new velocity sets:

  sum_i w_i = 1,  sum_i w_i c_ia c_ib = (5/9) delta_ab       (Eqs. 22, 24)
  sum_i h_i c_ia c_ib = delta_ab                             (Eq. 23)
  sum_i h_i c_ia c_ib c_ig c_id = (1/3)(d_ab d_gd + d_ag d_bd + d_ad d_bg)
                                                             (Eq. 25's source)
with h_i = 5 a_i / 3 the coefficient of c_i . q in Eq. 15.  On D3Q14
(6 axis + 8 corner velocities) they have one solution: w = 1/9, 1/24 and
h = 1/3, 1/24; the analysis of Eqs. 39-47 then returns Eq. 7 with the same
lattice speed c = sqrt(3/5) v_g (Eq. 48) and tau = tau_C + 1/2 (Eq. 49).
D1Q2 (c = +-1) forces w = h = 1/2; its second moment is c^2 e, so Eq. 38
gives c = v_g / sqrt(3), and the second moment of e^(1) vanishes: the scheme
recovers Eqs. 6-7 without the nonlocal term (the Cattaneo equation).

The step follows Eq. 13 in the paper's order on every node (Eqs. 53, 54,
15, 16), then push-streams each population to x + c_i on a periodic
lattice.  Populations are held as f[i, z, y, x] (x fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Lattice:
    name: str
    dim: int
    c: np.ndarray          # [Q, dim] integer velocities (lattice units)
    w: np.ndarray          # [Q] weights of C_V T in Eq. 15
    h: np.ndarray          # [Q] weights of c_i . q in Eqs. 15-16 (5 a_i / 3)
    speed: float           # lattice speed c / v_g

    @property
    def Q(self) -> int:
        return len(self.w)


def _d3q14():
    axis = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    # corners in opposite pairs: +-(1,1,1), +-(1,1,-1), +-(1,-1,1), +-(1,-1,-1)
    corner = []
    for b in ((1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)):
        corner += [b, tuple(-v for v in b)]
    c = np.array(axis + corner, dtype=np.int64)
    w = np.array([1 / 9] * 6 + [1 / 24] * 8)
    h = np.array([1 / 3] * 6 + [1 / 24] * 8)
    return Lattice("D3Q14", 3, c, w, h, math.sqrt(3 / 5))


D3Q14 = _d3q14()
D1Q2 = Lattice("D1Q2", 1, np.array([[1], [-1]], dtype=np.int64), np.array([0.5, 0.5]),
               np.array([0.5, 0.5]), 1 / math.sqrt(3))


def relaxation(tau_N: float, tau_R: float):
    """Section 2.1 and Eq. 49 in lattice steps: (tau, tau_r)."""
    inv_c = (0.0 if math.isinf(tau_N) else 1 / tau_N) + (0.0 if math.isinf(tau_R) else 1 / tau_R)
    return 1 / inv_c + 0.5, tau_R


def kappa(tau_r: float) -> float:
    """Eq. 54 prefactor 2 tau_r / (2 tau_r + 1) (1 when tau_r is infinite)."""
    return 1.0 if math.isinf(tau_r) else 2 * tau_r / (2 * tau_r + 1)


def _cdot(L: Lattice, q):
    """c_i . q for every i: array [Q, ...] from q = [dim, ...]."""
    return np.tensordot(L.c.astype(np.float64), q, axes=([1], [0]))


def moments(L: Lattice, f, tau_r):
    """Eqs. 53-54: e = sum_i f_i, q = kappa sum_i c_i f_i."""
    e = f.sum(0)
    q = kappa(tau_r) * np.tensordot(L.c.T.astype(np.float64), f, axes=([1], [0]))
    return e, q


def equilibrium(L: Lattice, e, q):
    """Eq. 15 with this lattice's weights."""
    shape = (L.Q,) + (1,) * np.ndim(e)
    return L.w.reshape(shape) * e + L.h.reshape((L.Q,) + (1,) * (np.ndim(q) - 1)) * _cdot(L, q)


def collide(L: Lattice, f, tau, tau_r):
    """Right-hand side of Eq. 13 with Eq. 16 (lattice form)."""
    e, q = moments(L, f, tau_r)
    eq = equilibrium(L, e, q)
    hq = L.h.reshape((L.Q,) + (1,) * (f.ndim - 1)) * _cdot(L, q)
    src = 0.0 if math.isinf(tau_r) else -(1 - 1 / (2 * tau)) * hq / tau_r
    return f + (eq - f) / tau + src


def stream(L: Lattice, f):
    """Push every population to x + c_i on the periodic lattice; f has the
    spatial axes (z, y, x) of the lattice's dimension after the i axis."""
    out = np.empty_like(f)
    for i in range(L.Q):
        # spatial axes are stored reversed (x last)
        shift = tuple(int(v) for v in L.c[i][::-1])
        out[i] = np.roll(f[i], shift, axis=tuple(range(L.dim)))
    return out


class Run:
    """A periodic lattice held by the oracle."""

    def __init__(self, L: Lattice, shape, tau_N, tau_R):
        self.L = L
        self.shape = tuple(shape)            # (nz, ny, nx) / (nx,)
        assert len(self.shape) == L.dim
        self.tau, self.tau_r = relaxation(tau_N, tau_R)
        self.f = np.zeros((L.Q,) + self.shape)
        self.step_count = 0

    def init(self, e, q=None):
        e = np.broadcast_to(np.asarray(e, dtype=np.float64), self.shape)
        q = np.zeros((self.L.dim,) + self.shape) if q is None else np.asarray(q, np.float64)
        self.f = equilibrium(self.L, e, q).copy()
        self.step_count = 0

    def step(self, n=1):
        for _ in range(int(n)):
            self.f = stream(self.L, collide(self.L, self.f, self.tau, self.tau_r))
        self.step_count += int(n)

    def moments(self):
        return moments(self.L, self.f, self.tau_r)


def mode_matrix(L: Lattice, k, tau, tau_r):
    """Exact one-step map of a Fourier mode f_i(x) = F_i exp(i k.x) on the
    periodic lattice (independent of the array code above): F(n+1) =
    diag(exp(-i k.c_i)) M F(n), M the collision matrix of Eqs. 13-16, 54."""
    c = L.c.astype(np.float64)
    kap = kappa(tau_r)
    cc = c @ c.T
    E = L.w[:, None] * np.ones((1, L.Q)) + L.h[:, None] * cc * kap
    S = np.zeros((L.Q, L.Q)) if math.isinf(tau_r) else \
        -(1 - 1 / (2 * tau)) * L.h[:, None] * cc * kap / tau_r
    M = np.eye(L.Q) + (E - np.eye(L.Q)) / tau + S
    phase = np.exp(-1j * (c @ np.asarray(k, dtype=np.float64)))
    return phase[:, None] * M
