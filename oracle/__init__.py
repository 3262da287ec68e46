"""FP64 CPU oracle for the phonon lattice Boltzmann scheme (Guo & Wang,
arXiv 2010.01847).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and imports nothing from it.

The arithmetic lives in ``phonon_lbm_oracle.c`` (plain C, FP64, the paper's
order of operations: collide by Eqs. 13/15/16/53/54, push-stream with the
Eq. 59-60 seam jump, then the Eq. 58 wall reflection).  This module only
loads it through ctypes and marshals numpy arrays.  ``update_matrix`` holds a
second, independent construction of the same linear map as explicit matrices
(tiny lattices only), used to pin the looped implementation.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, the paper's printed
relaxation times, brute-force matrices).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phonon_lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PERIODIC = 0
PERIODIC_GRADIENT = 1
WALLS = 2
SIDES = 3
# side treatments, sides numbered left, right, bottom, top
DIFFUSE, ISOTHERMAL, HEAT_FLUX = 0, 1, 2

# Eq. 14 in the order Eqs. 59-60 imply; index i = paper direction i+1.
CX = np.array([1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1])
# Eqs. 17 and 18.
OMEGA = np.array([2 / 9] * 4 + [1 / 36] * 4)
A_W = np.array([1 / 5] * 4 + [1 / 20] * 4)


def compile_library(src: str, out: str) -> str:
    """gcc the oracle source ``src`` into the shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle into ``liboracle.so`` next to its source."""
    if not force and os.path.exists(_LIB) and \
            os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_library(_SRC, _LIB)


_lib = None
_lib_path = None          # another build of the oracle (see use_library)


def use_library(path=None) -> None:
    """Point the module at another build of the oracle source (the tests
    that plant mistakes in the oracle use this); None returns to the
    regular ``liboracle.so``."""
    global _lib, _lib_path
    _lib, _lib_path = None, path


def _load():
    global _lib
    if _lib is None:
        if _lib_path is None:
            build()
        lib = ctypes.CDLL(_lib_path or _LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_tau_from_kn.restype = ctypes.c_double
        lib.orc_tau_from_kn.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_params.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        lib.orc_equilibrium.argtypes = [ctypes.c_double] * 3 + [dp]
        lib.orc_source.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.orc_node_moments.argtypes = [dp, ctypes.c_double, dp, dp, dp]
        lib.orc_collide_node.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_init.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, dp, ctypes.c_long]
        lib.orc_run_sides.restype = ctypes.c_int
        lib.orc_run_sides.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int), dp,
                                      ctypes.c_double, ctypes.c_double, dp, ctypes.c_long]
        lib.orc_moments.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    dp, dp, dp, dp]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return _load().orc_get_threads()


def tau_from_kn(kn: float, length: float) -> float:
    """Eq. 48: lattice relaxation time for Knudsen number ``kn`` over
    ``length`` cells (kn * length * sqrt(3/5))."""
    return _load().orc_tau_from_kn(float(kn), float(length))


def params(tau_N: float, tau_R: float) -> dict:
    """Eq. 49 and Section 2.4: tau, tau_r, tau_C from the two relaxation
    times (lattice units, math.inf allowed)."""
    out = np.zeros(3)
    _load().orc_params(float(tau_N), float(tau_R), _ptr(out))
    return {"tau": out[0], "tau_r": out[1], "tau_C": out[2]}


def equilibrium(e: float, qx: float, qy: float) -> np.ndarray:
    """Eq. 15 at one node."""
    out = np.zeros(8)
    _load().orc_equilibrium(float(e), float(qx), float(qy), _ptr(out))
    return out


def source(qx: float, qy: float, tau: float, tau_r: float) -> np.ndarray:
    """Eq. 16 times dt at one node."""
    out = np.zeros(8)
    _load().orc_source(float(qx), float(qy), float(tau), float(tau_r), _ptr(out))
    return out


def node_moments(f8: np.ndarray, tau_r: float):
    """Eqs. 53-54 at one node: (e, qx, qy)."""
    f8 = np.ascontiguousarray(f8, dtype=np.float64)
    e, qx, qy = (ctypes.c_double(), ctypes.c_double(), ctypes.c_double())
    _load().orc_node_moments(_ptr(f8), float(tau_r), ctypes.byref(e),
                             ctypes.byref(qx), ctypes.byref(qy))
    return e.value, qx.value, qy.value


def collide_node(f8: np.ndarray, tau: float, tau_r: float) -> np.ndarray:
    """Right-hand side of Eq. 13 at one node."""
    f8 = np.ascontiguousarray(f8, dtype=np.float64)
    out = np.zeros(8)
    _load().orc_collide_node(_ptr(f8), float(tau), float(tau_r), _ptr(out))
    return out


class Lattice:
    """A whole lattice held by the oracle: populations f[y, x, i] (AoS)."""

    def __init__(self, nx: int, ny: int, tau_N: float, tau_R: float,
                 bc_x: int = PERIODIC, bc_y: int = PERIODIC,
                 delta_e: float = 0.0, sides=None):
        self.nx, self.ny = int(nx), int(ny)
        self.tau_N, self.tau_R = float(tau_N), float(tau_R)
        self.bc_x, self.bc_y = int(bc_x), int(bc_y)
        self.delta_e = float(delta_e)
        self.f = np.zeros((self.ny, self.nx, 8))
        self.step_count = 0
        # [(kind, value)] x 4: left, right, bottom, top
        self.sides = list(sides) if sides is not None else [(DIFFUSE, 0.0)] * 4

    def set_side(self, side: int, kind: int, value: float = 0.0) -> None:
        self.sides[side] = (int(kind), float(value))

    def init(self, e, qx=None, qy=None) -> None:
        shape = (self.ny, self.nx)
        e = np.ascontiguousarray(np.broadcast_to(e, shape), dtype=np.float64)
        qx = np.zeros(shape) if qx is None else \
            np.ascontiguousarray(np.broadcast_to(qx, shape), dtype=np.float64)
        qy = np.zeros(shape) if qy is None else \
            np.ascontiguousarray(np.broadcast_to(qy, shape), dtype=np.float64)
        _load().orc_init(self.nx, self.ny, _ptr(e), _ptr(qx), _ptr(qy),
                         _ptr(self.f))
        self.step_count = 0

    def set_populations(self, f: np.ndarray) -> None:
        self.f = np.ascontiguousarray(f, dtype=np.float64).reshape(
            self.ny, self.nx, 8).copy()

    def step(self, n: int = 1) -> None:
        kinds = (ctypes.c_int * 4)(*[k for k, _ in self.sides])
        vals = np.array([v for _, v in self.sides], dtype=np.float64)
        rc = _load().orc_run_sides(self.nx, self.ny, self.bc_x, self.bc_y,
                                   self.delta_e, kinds, _ptr(vals), self.tau_N,
                                   self.tau_R, _ptr(self.f), int(n))
        if rc != 0:
            raise ValueError("oracle rejected the lattice parameters")
        self.step_count += int(n)

    def moments(self):
        """(e, qx, qy), each [ny, nx], of the current state (Eqs. 53-54)."""
        e = np.zeros((self.ny, self.nx))
        qx = np.zeros_like(e)
        qy = np.zeros_like(e)
        _load().orc_moments(self.nx, self.ny, self.tau_R, _ptr(self.f),
                            _ptr(e), _ptr(qx), _ptr(qy))
        return e, qx, qy


def run(nx, ny, tau_N, tau_R, e, qx=None, qy=None, steps=0,
        bc_x=PERIODIC, bc_y=PERIODIC, delta_e=0.0, sides=None):
    """Convenience: initialise, advance ``steps`` and return the lattice."""
    lat = Lattice(nx, ny, tau_N, tau_R, bc_x, bc_y, delta_e, sides)
    lat.init(e, qx, qy)
    if steps:
        lat.step(steps)
    return lat


def kappa(tau_r: float) -> float:
    """Eq. 54 prefactor (test helper mirroring the C definition)."""
    return 1.0 if math.isinf(tau_r) else 2 * tau_r / (2 * tau_r + 1)
