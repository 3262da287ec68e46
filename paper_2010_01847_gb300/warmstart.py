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
from . import analytic_profiles as _analytic

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


def _schedule(b, schedule):
    """Applies a batch schedule (None: the defaults; "tune": the autotuner,
    on the initialised batch; or a dict from schedule_of) before a solve."""
    if schedule == "tune":
        b.autotune(10)
    elif schedule:
        b.set_schedule(schedule["threads_per_item"], schedule["ctas_per_sm"])
        b.set_wave(schedule["wave_steps"], schedule["wave_rows"])


def schedule_of(b):
    """The schedule a batch runs with (to repeat it on another batch)."""
    s, w = b.schedule, b.wave
    return {"threads_per_item": s["threads_per_item"], "ctas_per_sm": s["ctas_per_sm"],
            "wave_steps": w["steps"], "wave_rows": w["rows"]}


def steady_profiles(instances, tol=1e-8, check_every=100, max_steps=400000, schedule=None,
                    start="cold"):
    """Solve every instance to steady state with the batched solver, from the
    cold start or (start="analytic") from the profile of Eq. 68, which
    converges to the same steady state in fewer steps; return (profiles
    [n, 512] CUDA tensor, steps, final residuals, seconds of the start and
    the solve)."""
    b = Batch(instances)
    b.init()
    _schedule(b, schedule)
    t0 = time.perf_counter()
    if start == "analytic":
        b.init_profiles(_analytic(instances))
    elif start != "cold":
        raise ValueError("start must be 'cold' or 'analytic'")
    steps, r = b.solve(tol, check_every, max_steps)
    dt = time.perf_counter() - t0
    prof = b.profiles()
    b.close()
    return prof, steps, r, dt


class WarmStart:
    """The network predicts the correction to the analytic profile (Eq. 68
    flux, uniform energy row profile) that takes it to the scheme's own
    steady state: the analytic part carries the physics the paper prints,
    the network what the discrete scheme adds (the walls' slip and Knudsen
    layers, the energy's row profile)."""

    def __init__(self, seed=0, max_batch=4096):
        self.net = Mlp(WIDTHS, max_batch=max_batch)
        self.net.init_params(seed)
        self.seed = seed

    def train(self, instances, profiles, steps=3000, batch=512, lr=1e-3, lr_final=1e-5):
        """Fits the network to (steady profiles - analytic profiles) of the
        training channels: Adam on minibatches drawn on the device with a
        seeded counter-based generator, cosine decay of the learning rate
        from lr to lr_final, all steps on the GPU (lbm_mlp_train).  Returns
        the loss history."""
        target = profiles.float().contiguous().clone()
        _analytic(instances, target, op=-1)
        return list(self.net.train(features(instances), target, steps, batch, lr, lr_final,
                                   seed=self.seed + 1))

    def predict(self, instances):
        """Profiles of the channels: the analytic ones plus the network's
        correction (CUDA tensor [n, 512])."""
        out = self.net.forward(features(instances)).contiguous()
        return _analytic(instances, out, op=1)


def solve(instances, profiles=None, tol=1e-8, check_every=100, max_steps=400000,
          schedule=None):
    """Batched solve from the cold start (profiles None) or from profiles
    (predicted, or analytic_profiles), with a schedule (see _schedule; set
    up before the timed solve); returns (steps, final residuals, seconds,
    batch)."""
    b = Batch(instances)
    if profiles is None:
        b.init()
    else:
        b.init_profiles(profiles)
    _schedule(b, schedule)
    t0 = time.perf_counter()
    steps, r = b.solve(tol, check_every, max_steps)
    return steps, r, time.perf_counter() - t0, b


def analytic_profiles(instances):
    """The analytic start of every channel: Q(Y) from Eq. 68, E(Y) = 0
    (lbm_analytic_profiles), as a CUDA tensor [n, 512]."""
    return _analytic(instances)


def shortened(instances, nx=TRAIN_NX):
    """The same channels with nx columns and the same temperature gradient
    (delta_e scaled by nx / nx_i).  A walled channel's steady state under the
    periodic gradient is the same at every x up to the affine part of e (q
    does not depend on x), so a short channel has the full one's steady
    rows."""
    return [dict(i, nx=nx, delta_e=i["delta_e"] * nx / i["nx"]) for i in instances]


def reference_profiles(instances, tol=1e-12, check_every=500, max_steps=4000000):
    """Steady profiles of the channels from FP64 storage solved to residual
    < tol on their shortened copies; returns (profiles CUDA tensor [n, 512],
    steps, residuals)."""
    short = shortened(instances)
    b = Batch(short, precision="fp64")
    b.init()
    steps, r = b.solve(tol, check_every, max_steps)
    prof = b.profiles()
    b.close()
    return prof, steps, r


def profile_errors(prof, ref, instances):
    """Errors of end-state profiles against reference profiles (both in the
    layout of lbm_batch_profiles, which depends on the gradient alone; ref
    from reference_profiles).  Per channel:
    err_q = max |Q - Q_ref| / max |Q_ref|; err_e = max over rows of the
    difference of e's departure from its x-affine part and row mean, over
    the largest |e - mean e| of the reference field (half the temperature
    drop plus the largest departure).  Returns two numpy arrays."""
    p = prof.double().cpu().numpy()
    r = ref.double().cpu().numpy()
    eq, ee = [], []
    for k, i in enumerate(instances):
        qg, qr = p[k, :256], r[k, :256]
        eq.append(np.abs(qg - qr).max() / np.abs(qr).max())
        drop = i["delta_e"] / i["nx"]          # both profiles: E in units of the drop per cell
        gg = (p[k, 256:] - p[k, 256:].mean()) * drop
        gr = (r[k, 256:] - r[k, 256:].mean()) * drop
        span = 0.5 * abs(i["delta_e"]) * (i["nx"] - 1) / i["nx"] + np.abs(gr).max()
        ee.append(np.abs(gg - gr).max() / span)
    return np.array(ee), np.array(eq)
