"""Explicit-matrix construction of one time step of the phonon LBM.

TEST INFRASTRUCTURE (part of the oracle).  This is a second, independent
construction of the same scheme as ``phonon_lbm_oracle.c``: instead of
looping over nodes it assembles

  * the 8x8 per-node collision matrix from Eqs. 13, 15, 16 and 54
    (post = M f, with M = I + (E - I)/tau + S),
  * the streaming/boundary map as a sparse affine matrix (Eq. 13 left-hand
    side, the seam jump of Eqs. 59-60, the diffuse wall of Eq. 58),

and composes them.  On tiny lattices ``step_matrix(...)^n`` applied to the
initial vector must equal the looped oracle after n steps (brute force).
``mode_matrix`` gives the exact one-step amplification matrix of a Fourier
mode exp(i k.x) on a periodic lattice.
"""
from __future__ import annotations

import math

import numpy as np

CX = np.array([1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1])
OMEGA = np.array([2 / 9] * 4 + [1 / 36] * 4)   # Eq. 17
A_W = np.array([1 / 5] * 4 + [1 / 20] * 4)     # Eq. 18


def collision_matrix(tau: float, tau_r: float) -> np.ndarray:
    """M with post_i = sum_j M_ij f_j (Eq. 13 right-hand side).

    e = sum_j f_j (Eq. 53); q = kappa sum_j c_j f_j (Eq. 54);
    e_i^eq = w_i e + (5/3) a_i c_i.q (Eq. 15);
    S_i = -(1 - 1/(2 tau)) (5/3) a_i c_i.q / tau_r (Eq. 16).
    """
    kap = 1.0 if math.isinf(tau_r) else 2 * tau_r / (2 * tau_r + 1)
    cc = np.outer(CX, CX) + np.outer(CY, CY)          # c_i . c_j
    E = OMEGA[:, None] * np.ones((1, 8)) + (5 / 3) * A_W[:, None] * cc * kap
    if math.isinf(tau_r):
        S = np.zeros((8, 8))
    else:
        S = -(1 - 1 / (2 * tau)) * (5 / 3) * A_W[:, None] * cc * kap / tau_r
    return np.eye(8) + (E - np.eye(8)) / tau + S


def mode_matrix(kx: float, ky: float, tau: float, tau_r: float) -> np.ndarray:
    """Exact one-step map of a Fourier mode f_i(x) = F_i exp(i k.x) on a
    periodic lattice: F(n+1) = diag(exp(-i k.c_i)) M F(n)."""
    phase = np.exp(-1j * (kx * CX + ky * CY))
    return phase[:, None] * collision_matrix(tau, tau_r)


def step_matrix(nx: int, ny: int, tau: float, tau_r: float, bc_x: int,
                bc_y: int, delta_e: float) -> np.ndarray:
    """Dense affine matrix T of size (8N+1)^2 acting on [f; 1], with
    f flattened as f[(y*nx + x)*8 + i] (the oracle's layout).

    bc codes: 0 periodic, 1 periodic temperature gradient (x only),
    2 diffuse adiabatic walls (y only).
    """
    n = nx * ny
    dim = 8 * n + 1
    M = collision_matrix(tau, tau_r)
    C = np.zeros((dim, dim))
    for s in range(n):
        C[8 * s:8 * s + 8, 8 * s:8 * s + 8] = M
    C[-1, -1] = 1.0

    # streaming: row = destination slot, column = source slot
    P = np.zeros((dim, dim))
    P[-1, -1] = 1.0
    for y in range(ny):
        for x in range(nx):
            for i in range(8):
                ty, tx = y + CY[i], x + CX[i]
                if not 0 <= ty < ny:
                    if bc_y == 2:
                        continue
                    ty %= ny
                jump = 0.0
                if not 0 <= tx < nx:
                    if bc_x == 1:
                        jump = OMEGA[i] * delta_e * (1 if tx >= nx else -1)
                    tx %= nx
                dst = 8 * (ty * nx + tx) + i
                P[dst, 8 * (y * nx + x) + i] = 1.0
                P[dst, -1] += jump

    # Eq. 58 at wall rows: unknown = w_i / sum_leaving(w) * sum incident
    B = np.eye(dim)
    if bc_y == 2:
        for y, n_y in ((0, -1), (ny - 1, 1)):
            incident = [i for i in range(8) if CY[i] * n_y > 0]
            leaving = [i for i in range(8) if CY[i] * n_y < 0]
            w_leave = OMEGA[leaving].sum()
            for x in range(nx):
                base = 8 * (y * nx + x)
                for i in leaving:
                    B[base + i, :] = 0.0
                    for j in incident:
                        B[base + i, base + j] = OMEGA[i] / w_leave
    return B @ P @ C
