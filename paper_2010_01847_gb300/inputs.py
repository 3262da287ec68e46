"""Seeded synthetic input fields and the workload table.

This module holds no arithmetic of the lattice Boltzmann method: it only
produces initial energy-density / heat-flux fields (numpy float64, shape
[ny, nx], index [y, x]) and names the workloads by their sizes, Knudsen
numbers and boundary kinds.  Both the CUDA path and the FP64 oracle read the
same arrays, so neither side generates inputs for the other.

Noise is a counter-based generator: SplitMix64 of (seed XOR site index),
top 53 bits mapped to [0, 1), then scaled to [-amp, +amp).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# boundary kinds (same numbering as the C-ABI)
PERIODIC = 0
PERIODIC_GRADIENT = 1
WALLS = 2

SEED = 201001847

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_noise(shape, amp: float, seed: int = SEED,
                  offset: int = 0) -> np.ndarray:
    """i.i.d. U[-amp, amp) per site; site s = y*nx + x (+offset)."""
    n = int(np.prod(shape))
    idx = np.arange(offset, offset + n, dtype=np.uint64) ^ np.uint64(seed)
    u = (splitmix64(idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (amp * (2.0 * u - 1.0)).reshape(shape)


def uniform_field(nx: int, ny: int, e0: float = 1.0) -> np.ndarray:
    return np.full((ny, nx), float(e0))


def sine_mode(nx: int, ny: int, wavelength: float, amplitude: float,
              e0: float = 1.0, noise: float = 0.0, seed: int = SEED,
              direction: str = "x") -> np.ndarray:
    """e = e0 + amplitude sin(2 pi s / wavelength) (+ uniform noise), s = x,
    y or x+y depending on ``direction``."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = {"x": x, "y": y, "xy": x + y}[direction]
    e = e0 + amplitude * np.sin(2.0 * np.pi * s / wavelength)
    if noise:
        e = e + uniform_noise((ny, nx), noise, seed)
    return e


def gaussian_pulse(nx: int, ny: int, center: float, sigma: float,
                   amplitude: float, e0: float = 1.0) -> np.ndarray:
    """e = e0 + amplitude exp(-(x - center)^2 / (2 sigma^2)), uniform in y."""
    x = np.arange(nx, dtype=np.float64)
    prof = e0 + amplitude * np.exp(-((x - center) ** 2) / (2.0 * sigma ** 2))
    return np.broadcast_to(prof, (ny, nx)).copy()


def random_state_fields(nx: int, ny: int, seed: int = SEED, e0: float = 1.0,
                        amp: float = 1e-3):
    """Generic seeded (e, qx, qy) fields with structure at every scale,
    for parity tests: e = e0 + noise, q = noise of the same size."""
    e = e0 + uniform_noise((ny, nx), amp, seed, 0)
    qx = uniform_noise((ny, nx), amp, seed, 1 << 40)
    qy = uniform_noise((ny, nx), amp, seed, 2 << 40)
    return e, qx, qy


@dataclass(frozen=True)
class Workload:
    """A named workload: lattice, Knudsen numbers with their length, steps."""
    name: str
    nx: int
    ny: int
    kn_N: float
    kn_R: float
    length: float          # characteristic length (cells) of the Kn numbers
    steps: int
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    delta_e: float = 0.0
    extra: dict = field(default_factory=dict)


# Phonon Poiseuille channel: 128x32, periodic temperature gradient along x,
# diffuse walls at y = 0 and 31 (d = 31 cells), uniform start.
POISEUILLE_128x32 = Workload("poiseuille_128x32", 128, 32, 0.01, 1.0, 31.0,
                             10000, PERIODIC_GRADIENT, WALLS, 1e-3)

# Second-sound pulse: 4096x4 periodic, Gaussian pulse (amplitude 1e-3,
# width 20 cells); Kn measured on the 4096-cell period.
def second_sound_4096x4(kn_R: float) -> Workload:
    return Workload(f"second_sound_4096x4_knR{kn_R:g}", 4096, 4, 1e-3, kn_R,
                    4096.0, 5000)

# Large 2-D heat transport: 8192x8192 periodic, sine mode of wavelength 512
# plus U[-1e-6, 1e-6) noise; Kn measured on the 512-cell wavelength.
THROUGHPUT_8192 = Workload("heat_mode_8192x8192", 8192, 8192, 0.01, 0.1,
                           512.0, 2000)


def initial_fields(w: Workload):
    """(e, qx, qy) initial fields of a named workload (q = 0 throughout)."""
    if w.name.startswith("poiseuille"):
        e = uniform_field(w.nx, w.ny)
    elif w.name.startswith("second_sound"):
        e = gaussian_pulse(w.nx, w.ny, w.nx / 2, 20.0, 1e-3)
    elif w.name.startswith("heat_mode"):
        e = sine_mode(w.nx, w.ny, 512.0, 1e-3, noise=1e-6)
    else:
        raise KeyError(w.name)
    z = np.zeros_like(e)
    return e, z, z.copy()


def batch_channels(count: int, seed: int = SEED, w_range=(16, 512),
                   kn_N_range=(1e-3, 1e-1), kn_R_range=(0.1, 10.0)):
    """Candidate phonon-Poiseuille channels for the batched workload: width W
    uniform in w_range (integers), length 4W, Kn_N and Kn_R log-uniform,
    seeded.  Returns a list of dicts (W, nx=4W, ny=W, kn_N, kn_R, d=W-1);
    the caller decides which candidates it keeps."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        W = int(rng.integers(w_range[0], w_range[1] + 1))
        kn_N = float(10 ** rng.uniform(np.log10(kn_N_range[0]), np.log10(kn_N_range[1])))
        kn_R = float(10 ** rng.uniform(np.log10(kn_R_range[0]), np.log10(kn_R_range[1])))
        out.append({"W": W, "nx": 4 * W, "ny": W, "kn_N": kn_N, "kn_R": kn_R, "d": W - 1})
    return out
