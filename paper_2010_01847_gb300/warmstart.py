"""Learned warm start for batched channel solves.

A network (3 inputs -> 4 x 256 GELU -> 512) maps a channel's parameters
(tau_N, tau_R, width W) to its normalised steady profile (256 points of the
heat flux over the Fourier flux and 256 of the energy profile, the layout of
lbm_batch_profiles).  Training data are steady states computed by the
batched solver itself; the network is trained on the GPU by its own BF16
kernels; a solve starts from the predicted profile (lbm_batch_init_profiles)
and the plain solver always runs to the residual tolerance from there, so
the network only changes where the solve starts, never its end criterion.

The steady state of a channel with the periodic temperature gradient is
invariant along x (q) and affine in x (e), for any channel length, so the
training channels use the shortest length the vector layout allows
(nx = 8); profiles are normalised so they do not depend on the length.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import Batch, Mlp, inputs, tau_from_kn

WIDTHS = (3, 256, 256, 256, 256, 512)
TRAIN_NX = 8
# feature ranges (log10) used to scale the inputs to about [-1, 1]
_LOG_RANGES = ((-2.0, 1.7), (0.0, 3.7), (1.2, 2.8))


def channels(n, seed, nx=None, w_range=(16, 512), tau_min=0.6, delta_e=1e-3):
    """Seeded channel instances (walls, periodic gradient), keeping those
    whose tau is at least tau_min (the scheme's linear-stability bound with
    margin).  nx=None keeps the candidates' length 4W."""
    out = []
    for c in inputs.batch_channels(8 * n, seed=seed, w_range=w_range):
        tau_N = tau_from_kn(c["kn_N"], c["d"])
        tau_R = tau_from_kn(c["kn_R"], c["d"])
        if 1.0 / (1.0 / tau_N + 1.0 / tau_R) + 0.5 < tau_min:
            continue
        out.append(dict(nx=nx or c["nx"], ny=c["ny"], tau_N=tau_N, tau_R=tau_R,
                        bc_x=inputs.PERIODIC_GRADIENT, bc_y=inputs.WALLS, delta_e=delta_e,
                        W=c["W"], kn_N=c["kn_N"], kn_R=c["kn_R"]))
        if len(out) == n:
            break
    return out


def features(instances):
    """Network inputs: log10 of tau_N, tau_R and W, scaled to about [-1, 1]."""
    raw = np.array([[math.log10(i["tau_N"]), math.log10(i["tau_R"]), math.log10(i["ny"])]
                    for i in instances])
    lo = np.array([r[0] for r in _LOG_RANGES])
    hi = np.array([r[1] for r in _LOG_RANGES])
    return (2.0 * (raw - lo) / (hi - lo) - 1.0).astype(np.float32)


def steady_profiles(instances, tol=1e-8, check_every=100, max_steps=400000):
    """Solve every instance to steady state (cold start) with the batched
    solver and return (profiles [n, 512] CUDA tensor, steps, seconds)."""
    b = Batch(instances)
    b.init()
    t0 = time.perf_counter()
    steps, r = b.solve(tol, check_every, max_steps)
    dt = time.perf_counter() - t0
    prof = b.profiles()
    b.close()
    return prof, steps, r, dt


class WarmStart:
    def __init__(self, seed=0, max_batch=4096):
        self.net = Mlp(WIDTHS, max_batch=max_batch)
        self.net.init_params(seed)
        self.seed = seed

    def train(self, x, y, steps=3000, batch=512, lr=1e-3, lr_final=1e-5):
        """Adam on minibatches drawn with a seeded generator; cosine decay of
        the learning rate.  Returns the loss history."""
        rng = np.random.default_rng(self.seed + 1)
        xd = self.net._dev(x)
        yd = self.net._dev(y)
        n = xd.shape[0]
        hist = []
        for s in range(steps):
            idx = self.net.torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False),
                                           device="cuda")
            lr_s = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / steps))
            hist.append(self.net.train_step(xd[idx], yd[idx], lr_s))
        return hist

    def predict(self, instances):
        return self.net.forward(features(instances))


def solve(instances, profiles=None, tol=1e-8, check_every=100, max_steps=400000):
    """Batched solve from the cold start (profiles None) or from predicted
    profiles; returns (steps, final residuals, seconds, batch)."""
    b = Batch(instances)
    if profiles is None:
        b.init()
    else:
        b.init_profiles(profiles)
    t0 = time.perf_counter()
    steps, r = b.solve(tol, check_every, max_steps)
    return steps, r, time.perf_counter() - t0, b
