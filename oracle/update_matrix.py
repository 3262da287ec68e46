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
                bc_y: int, delta_e: float, sides=None) -> np.ndarray:
    """Dense affine matrix T of size (8N+1)^2 acting on [f; 1], with
    f flattened as f[(y*nx + x)*8 + i] (the oracle's layout).

    bc codes: 0 periodic, 1 periodic temperature gradient (x only),
    2 diffuse adiabatic walls (y only), 3 per-side treatments ``sides`` =
    [(kind, value)] for left, right, bottom, top with kind 0 diffuse
    (Eq. 58), 1 isothermal at e_s = value (Eq. 55), 2 incident heat flux
    q_0 = value (Eq. 57).
    """
    sides = sides or [(0, 0.0)] * 4
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
                    if bc_y in (2, 3):
                        continue
                    ty %= ny
                jump = 0.0
                if not 0 <= tx < nx:
                    if bc_x == 3:
                        continue
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
    T = B @ P @ C
    if bc_x == 3 or bc_y == 3:
        kap = 1.0 if math.isinf(tau_r) else 2 * tau_r / (2 * tau_r + 1)
        normals = [(-1, 0), (1, 0), (0, -1), (0, 1)]
        for y in range(ny):
            for x in range(nx):
                on = [bc_x == 3 and x == 0, bc_x == 3 and x == nx - 1,
                      bc_y == 3 and y == 0, bc_y == 3 and y == ny - 1]
                if not any(on):
                    continue
                base = 8 * (y * nx + x)
                iso = [sd for sd in range(4) if on[sd] and sides[sd][0] == 1]
                S = np.eye(dim)
                if iso:
                    # Eq. 55: node at equilibrium at rest at e_s
                    for i in range(8):
                        S[base + i, :] = 0.0
                        S[base + i, -1] = OMEGA[i] * sides[iso[0]][1]
                    T = S @ T
                    continue
                for sd in (2, 3, 0, 1):
                    if not on[sd]:
                        continue
                    nxo, nyo = normals[sd]
                    cn = CX * nxo + CY * nyo
                    inc = [i for i in range(8) if cn[i] > 0]
                    lev = [i for i in range(8) if cn[i] < 0]
                    wl = OMEGA[lev].sum()
                    q0 = sides[sd][1] if sides[sd][0] == 2 else 0.0
                    S = np.eye(dim)
                    for i in lev:
                        S[base + i, :] = 0.0
                        for j in inc:
                            S[base + i, base + j] = OMEGA[i] / wl
                        S[base + i, -1] = OMEGA[i] / wl * q0 / kap
                    T = S @ T
    return T
