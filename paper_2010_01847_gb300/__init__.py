"""GB300 (sm_103a) phonon lattice Boltzmann solver - Python binding.

The solver advances Guo & Wang's lattice Boltzmann scheme for the phonon
Boltzmann equation under Callaway's dual relaxation model (arXiv
2010.01847, Section 2) on a D2Q8 lattice.  Every step of the method runs in
the CUDA kernels of ``libphonon_lbm.so`` behind the C-ABI declared in
``include/phonon_lbm.h``; this module only marshals arguments through
ctypes.  PyTorch supplies device memory (the two population buffers) and the
CUDA stream.  There is no CPU fallback: without the compiled library or a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphonon_lbm.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED = range(7)
PERIODIC, PERIODIC_GRADIENT, DIFFUSE_WALLS, SIDES = 0, 1, 2, 3
LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3                 # sides (lbm_side)
DIFFUSE, ISOTHERMAL, HEAT_FLUX = 0, 1, 2              # side treatments (lbm_side_kind)
FP32, FP16_DEV, BF16_DEV, FP64 = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_SCALAR, KERNEL_VECTOR, KERNEL_STAGED, KERNEL_RESIDENT, KERNEL_WAVE = range(6)
TIMED_WAVE, TIMED_SINGLE, TIMED_RESIDUAL = 0, 1, 2     # lbm_timed

D1Q2, D3Q14 = 1, 3                                     # lbm_lattice
PRECISIONS = {"fp32": FP32, "fp16": FP16_DEV, "bf16": BF16_DEV, "fp64": FP64}
ROUND_NEAREST, ROUND_STOCHASTIC = 0, 1
ROUNDINGS = {"nearest": ROUND_NEAREST, "stochastic": ROUND_STOCHASTIC}
KERNELS = {"auto": KERNEL_AUTO, "scalar": KERNEL_SCALAR, "vector": KERNEL_VECTOR,
           "staged": KERNEL_STAGED, "resident": KERNEL_RESIDENT, "wave": KERNEL_WAVE}
_ELEM = {FP32: 4, FP16_DEV: 2, BF16_DEV: 2, FP64: 8}

# Every symbol include/phonon_lbm.h declares.
EXPORTS = [
    "lbm_tau_from_kn", "lbm_population_bytes", "lbm_create", "lbm_create_ex",
    "lbm_destroy", "lbm_init", "lbm_init_device", "lbm_step", "lbm_sync",
    "lbm_moments", "lbm_moments_device", "lbm_populations", "lbm_residual",
    "lbm_step_residual",
    "lbm_state_bytes", "lbm_get_state", "lbm_set_state", "lbm_step_count",
    "lbm_set_kernel", "lbm_get_kernel", "lbm_set_side", "lbm_get_side",
    "lbm_set_staged_config", "lbm_get_staged_config", "lbm_set_rounding",
    "lbm_set_graph_chunk", "lbm_autotune", "lbm_set_wave_config", "lbm_get_wave_config",
    "lbm_set_launch_timing", "lbm_launch_time",
    "lbm_kernel_launches", "lbm_storage_scale", "lbm_last_error",
    "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_init", "lbm_batch_step",
    "lbm_batch_residuals", "lbm_batch_solve", "lbm_batch_moments", "lbm_batch_set_schedule",
    "lbm_batch_get_schedule", "lbm_batch_autotune", "lbm_batch_active", "lbm_batch_steps",
    "lbm_batch_set_wave", "lbm_batch_get_wave",
    "lbm_batch_last_error", "lbm_batch_profiles", "lbm_batch_init_profiles",
    "lbm_analytic_profiles",
    "lbm_mlp_create", "lbm_mlp_destroy", "lbm_mlp_param_count", "lbm_mlp_set_params",
    "lbm_mlp_get_params", "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_train_step",
    "lbm_mlp_train", "lbm_mlp_last_error",
    "lbm_residual_noalloc", "lbm_check_bounded_wait", "lbm_probe_resident_wait",
    "lbm_nd_lattice_speed", "lbm_nd_create", "lbm_nd_init", "lbm_nd_step", "lbm_nd_sync",
    "lbm_nd_moments", "lbm_nd_populations", "lbm_nd_energy", "lbm_nd_step_count",
    "lbm_nd_destroy", "lbm_nd_last_error",
]
NOALLOC_MAX_NODES = 16777216


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[lbm status {status}] {message}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int)]


class Boundary(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int), ("y", ctypes.c_int), ("delta_e", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau_N", ctypes.c_double),
                ("tau_R", ctypes.c_double), ("bc", Boundary)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the compiled C-ABI library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; "
            "g.build()'` (the CUDA path has no fallback)")
    lib = ctypes.CDLL(path)
    vp, dp, c_long, c_size = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), \
        ctypes.c_long, ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "lbm_tau_from_kn": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
        "lbm_population_bytes": (c_size, [Grid, ctypes.c_int]),
        "lbm_create": (st, [Grid, ctypes.c_double, ctypes.c_double, Boundary, ctypes.c_int,
                            ctypes.c_double, vp, ctypes.POINTER(vp)]),
        "lbm_create_ex": (st, [Grid, ctypes.c_double, ctypes.c_double, Boundary, ctypes.c_int,
                               ctypes.c_double, vp, vp, vp, c_size, ctypes.POINTER(vp)]),
        "lbm_destroy": (None, [vp]),
        "lbm_init": (st, [vp, dp, dp, dp]),
        "lbm_init_device": (st, [vp, vp, vp, vp]),
        "lbm_step": (st, [vp, c_long]),
        "lbm_sync": (st, [vp]),
        "lbm_moments": (st, [vp, dp, dp, dp]),
        "lbm_moments_device": (st, [vp, vp, vp, vp]),
        "lbm_populations": (st, [vp, dp]),
        "lbm_residual": (st, [vp, dp, dp]),
        "lbm_step_residual": (st, [vp, c_long, dp, dp]),
        "lbm_state_bytes": (c_size, [vp]),
        "lbm_get_state": (st, [vp, vp, c_size]),
        "lbm_set_state": (st, [vp, vp, c_size]),
        "lbm_step_count": (c_long, [vp]),
        "lbm_set_kernel": (st, [vp, ctypes.c_int]),
        "lbm_get_kernel": (ctypes.c_int, [vp]),
        "lbm_set_side": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
        "lbm_get_side": (st, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]),
        "lbm_set_graph_chunk": (st, [vp, ctypes.c_int]),
        "lbm_autotune": (st, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]),
        "lbm_set_wave_config": (st, [vp, ctypes.c_int, ctypes.c_int]),
        "lbm_get_wave_config": (st, [vp, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
        "lbm_set_launch_timing": (st, [vp, ctypes.c_int]),
        "lbm_launch_time": (st, [vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong)]),
        "lbm_set_rounding": (st, [vp, ctypes.c_int]),
        "lbm_set_staged_config": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int]),
        "lbm_get_staged_config": (st, [vp] + [ctypes.POINTER(ctypes.c_int)] * 5),
        "lbm_kernel_launches": (ctypes.c_longlong, [vp]),
        "lbm_storage_scale": (ctypes.c_double, [vp]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_batch_create": (st, [ctypes.POINTER(Instance), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, vp, ctypes.POINTER(vp)]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_init": (st, [vp, dp, dp, dp]),
        "lbm_batch_step": (st, [vp, c_long]),
        "lbm_batch_residuals": (st, [vp, dp, dp]),
        "lbm_batch_solve": (st, [vp, ctypes.c_double, ctypes.c_int, c_long,
                                 ctypes.POINTER(c_long), dp]),
        "lbm_batch_moments": (st, [vp, ctypes.c_int, dp, dp, dp]),
        "lbm_batch_set_schedule": (st, [vp, ctypes.c_int, ctypes.c_int]),
        "lbm_batch_get_schedule": (st, [vp] + [ctypes.POINTER(ctypes.c_int)] * 3),
        "lbm_batch_autotune": (st, [vp, ctypes.c_int, dp]),
        "lbm_batch_set_wave": (st, [vp, ctypes.c_int, ctypes.c_int]),
        "lbm_batch_get_wave": (st, [vp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_active": (c_long, [vp]),
        "lbm_batch_steps": (c_long, [vp, ctypes.c_int]),
        "lbm_batch_last_error": (ctypes.c_char_p, [vp]),
        "lbm_batch_profiles": (st, [vp, vp]),
        "lbm_batch_init_profiles": (st, [vp, vp]),
        "lbm_analytic_profiles": (st, [vp, ctypes.c_int, vp, ctypes.c_int, vp]),
        "lbm_mlp_create": (st, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, vp,
                                ctypes.POINTER(vp)]),
        "lbm_mlp_destroy": (None, [vp]),
        "lbm_mlp_param_count": (c_size, [vp]),
        "lbm_mlp_set_params": (st, [vp, vp]),
        "lbm_mlp_get_params": (st, [vp, vp]),
        "lbm_mlp_forward": (st, [vp, vp, ctypes.c_int, vp]),
        "lbm_mlp_loss_grad": (st, [vp, vp, vp, ctypes.c_int, dp, vp]),
        "lbm_mlp_train_step": (st, [vp, vp, vp, ctypes.c_int, ctypes.c_float, dp]),
        "lbm_mlp_train": (st, [vp, vp, vp, ctypes.c_int, ctypes.c_int, c_long, ctypes.c_float,
                               ctypes.c_float, ctypes.c_ulonglong, vp]),
        "lbm_mlp_last_error": (ctypes.c_char_p, [vp]),
        "lbm_residual_noalloc": (st, [vp, vp, vp, vp, vp, vp, ctypes.c_longlong,
                                      ctypes.c_double, c_long, vp, dp, dp]),
        "lbm_check_bounded_wait": (st, [vp, ctypes.POINTER(ctypes.c_int), dp]),
        "lbm_probe_resident_wait": (st, [vp]),
        "lbm_nd_lattice_speed": (ctypes.c_double, [ctypes.c_int]),
        "lbm_nd_create": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                               vp, ctypes.POINTER(vp)]),
        "lbm_nd_init": (st, [vp, dp, dp]),
        "lbm_nd_step": (st, [vp, c_long]),
        "lbm_nd_sync": (st, [vp]),
        "lbm_nd_moments": (st, [vp, dp, dp]),
        "lbm_nd_populations": (st, [vp, dp]),
        "lbm_nd_energy": (st, [vp, dp]),
        "lbm_nd_step_count": (c_long, [vp]),
        "lbm_nd_destroy": (None, [vp]),
        "lbm_nd_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def tau_from_kn(kn: float, length: float) -> float:
    """Eq. 48 in lattice units: kn * length * sqrt(3/5)."""
    return load_library().lbm_tau_from_kn(float(kn), float(length))


def residual_noalloc(fields, prev_fields=None, k_steps=0, e_ref=1.0, stream=None):
    """lbm_residual_noalloc on CUDA float64 tensors: (r, total energy).
    ``fields`` / ``prev_fields`` are (e, qx, qy) of equal size; the call
    allocates no device memory."""
    lib = load_library()
    e, qx, qy = fields
    n = e.numel()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    prev = [ptr(t) for t in prev_fields] if prev_fields is not None else [None] * 3
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    r, en = ctypes.c_double(), ctypes.c_double()
    st = lib.lbm_residual_noalloc(ptr(e), ptr(qx), ptr(qy), *prev, n, float(e_ref),
                                  int(k_steps), ctypes.c_void_p(stream), ctypes.byref(r),
                                  ctypes.byref(en))
    if st != OK:
        raise LBMError(st, lib.lbm_last_error(None).decode())
    return r.value, en.value


def check_bounded_wait(stream=None):
    """lbm_check_bounded_wait: (gave_up, seconds) of the staged kernel's
    bounded mbarrier wait run against a barrier nothing completes."""
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    g, sec = ctypes.c_int(), ctypes.c_double()
    st = lib.lbm_check_bounded_wait(ctypes.c_void_p(stream), ctypes.byref(g), ctypes.byref(sec))
    if st != OK:
        raise LBMError(st, lib.lbm_last_error(None).decode())
    return bool(g.value), sec.value


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Lattice:
    """One D2Q8 lattice on one GPU.

    Parameters are in lattice units: ``tau_N``, ``tau_R`` are relaxation
    times in steps (``math.inf`` allowed for one of them); ``bc_x`` is
    PERIODIC, PERIODIC_GRADIENT (with ``delta_e`` = e_h - e_c of
    Eqs. 59-60) or SIDES, ``bc_y`` is PERIODIC, DIFFUSE_WALLS (Eq. 58) or
    SIDES.  The sides of a SIDES direction are set by ``sides`` (a list of
    four (kind, value) pairs for LEFT, RIGHT, BOTTOM, TOP, or a dict
    {side: (kind, value)}) or by ``set_side``; see lbm_set_side.
    ``precision`` is one of "fp32", "fp16", "bf16", "fp64".
    """

    def __init__(self, nx, ny, tau_N, tau_R, bc_x=PERIODIC, bc_y=PERIODIC, delta_e=0.0,
                 precision="fp32", e_ref=1.0, kernel="auto", device=None,
                 torch_buffers=True, graph_chunk=None, sides=None, buffers=None,
                 rounding="nearest"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the phonon LBM runs only on the GPU")
        self._lib = load_library()
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else device)
        self.nx, self.ny = int(nx), int(ny)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._ctx = ctypes.c_void_p()
        grid = Grid(self.nx, self.ny)
        bc = Boundary(int(bc_x), int(bc_y), float(delta_e))
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            sp = ctypes.c_void_p(self.stream.cuda_stream)
            if torch_buffers or buffers is not None:
                nbytes = self._lib.lbm_population_bytes(grid, self.precision)
                if nbytes == 0:
                    raise LBMError(EINVAL, "invalid grid or precision")
                if buffers is not None:
                    # caller-owned CUDA tensors (e.g. views into a larger allocation)
                    self._bufs = list(buffers)
                    nbytes = min(b.numel() * b.element_size() for b in self._bufs)
                else:
                    self._bufs = [torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                                  for _ in range(2)]
                st = self._lib.lbm_create_ex(grid, float(tau_N), float(tau_R), bc,
                                             self.precision, float(e_ref), sp,
                                             ctypes.c_void_p(self._bufs[0].data_ptr()),
                                             ctypes.c_void_p(self._bufs[1].data_ptr()),
                                             nbytes, ctypes.byref(self._ctx))
            else:
                self._bufs = []
                st = self._lib.lbm_create(grid, float(tau_N), float(tau_R), bc, self.precision,
                                          float(e_ref), sp, ctypes.byref(self._ctx))
        if st != OK:
            self._ctx = ctypes.c_void_p()
            raise LBMError(st, self._lib.lbm_last_error(None).decode())
        if sides is not None:
            items = sides.items() if isinstance(sides, dict) else enumerate(sides)
            for side, (kind, value) in items:
                if kind is not None:
                    self.set_side(side, kind, value)
        if kernel != "auto":
            self.set_kernel(kernel)
        if graph_chunk is not None:
            self._check(self._lib.lbm_set_graph_chunk(self._ctx, int(graph_chunk)))
        if rounding != "nearest":
            self.set_rounding(rounding)

    def set_rounding(self, rounding: str):
        """lbm_set_rounding: "nearest" or "stochastic" (16-bit storage)."""
        self._check(self._lib.lbm_set_rounding(self._ctx, ROUNDINGS[rounding]))

    # -- plumbing -----------------------------------------------------------
    def _check(self, st):
        if st != OK:
            raise LBMError(st, self._lib.lbm_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            self._lib.lbm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()
        self._bufs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._ctx

    # -- the solver ---------------------------------------------------------
    def init(self, e, qx=None, qy=None):
        """Step 0 = equilibrium of Eq. 15 from (e, q).  Host numpy arrays
        (or scalars) of shape [ny, nx], or CUDA float64 tensors."""
        torch = self.torch
        if isinstance(e, torch.Tensor) and e.is_cuda:
            def dev(a):
                if a is None:
                    return None
                a = a.to(device=self.device, dtype=torch.float64).contiguous()
                assert a.numel() == self.nx * self.ny
                return a
            e, qx, qy = dev(e), dev(qx), dev(qy)
            self._keep = (e, qx, qy)
            ptr = lambda a: ctypes.c_void_p(a.data_ptr()) if a is not None else None
            self._check(self._lib.lbm_init_device(self._ctx, ptr(e), ptr(qx), ptr(qy)))
            return
        shape = (self.ny, self.nx)
        host = lambda a: None if a is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
        e, qx, qy = host(e), host(qx), host(qy)
        p = lambda a: _dptr(a) if a is not None else None
        self._check(self._lib.lbm_init(self._ctx, p(e), p(qx), p(qy)))

    def step(self, n: int = 1):
        self._check(self._lib.lbm_step(self._ctx, int(n)))

    def set_side(self, side: int, kind: int, value: float = 0.0):
        """Treatment of one side of a SIDES direction (lbm_set_side):
        DIFFUSE (Eq. 58), ISOTHERMAL at e_s = value (Eq. 55) or HEAT_FLUX
        with incident flux q_0 = value (Eq. 57)."""
        self._check(self._lib.lbm_set_side(self._ctx, int(side), int(kind), float(value)))

    def side(self, side: int):
        """(kind, value) of one side."""
        k, v = ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.lbm_get_side(self._ctx, int(side), ctypes.byref(k),
                                           ctypes.byref(v)))
        return k.value, v.value

    def sync(self):
        self._check(self._lib.lbm_sync(self._ctx))

    def probe_resident_wait(self):
        """lbm_probe_resident_wait: runs the cluster-resident kernel's bounded
        ghost wait against a barrier nothing completes (about 2 s, async);
        the next synchronising call raises LBMError(ETIMEOUT)."""
        self._check(self._lib.lbm_probe_resident_wait(self._ctx))

    def moments(self, out=None):
        """(e, qx, qy) of the current state as numpy [ny, nx] float64.
        ``out``: three C-contiguous float64 arrays of that shape to fill
        (e.g. views of pinned host memory, so the copy runs at full speed)."""
        if out is None:
            out = [np.empty((self.ny, self.nx)) for _ in range(3)]
        for a in out:
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != self.nx * self.ny:
                raise ValueError("out arrays must be C-contiguous float64 of ny*nx elements")
        e, qx, qy = out
        self._check(self._lib.lbm_moments(self._ctx, _dptr(e), _dptr(qx), _dptr(qy)))
        return e, qx, qy

    def moments_device(self, out=None):
        """(e, qx, qy) as CUDA float64 tensors [ny, nx] (async)."""
        torch = self.torch
        if out is None:
            out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
                   for _ in range(3)]
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in out]
        self._check(self._lib.lbm_moments_device(self._ctx, *ptrs))
        return out

    def populations(self):
        """Raw populations e_i of the current state, numpy [8, ny, nx]."""
        f = np.empty((8, self.ny, self.nx))
        self._check(self._lib.lbm_populations(self._ctx, _dptr(f)))
        return f

    def residual(self):
        """(r, total energy): FP64 device reduction (see lbm_residual)."""
        r, en = ctypes.c_double(), ctypes.c_double()
        st = self._lib.lbm_residual(self._ctx, ctypes.byref(r), ctypes.byref(en))
        self._check(st)
        return r.value, en.value

    def step_residual(self, n: int):
        """Advance n steps; (r, total energy) of the final state, reduced
        inside the last step's launch (see lbm_step_residual)."""
        r, en = ctypes.c_double(), ctypes.c_double()
        st = self._lib.lbm_step_residual(self._ctx, int(n), ctypes.byref(r), ctypes.byref(en))
        self._check(st)
        return r.value, en.value

    def get_state(self) -> bytes:
        n = self._lib.lbm_state_bytes(self._ctx)
        buf = ctypes.create_string_buffer(n)
        self._check(self._lib.lbm_get_state(self._ctx, buf, n))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self._lib.lbm_set_state(self._ctx, buf, len(blob)))

    @property
    def step_count(self) -> int:
        return self._lib.lbm_step_count(self._ctx)

    @property
    def kernel_launches(self) -> int:
        return self._lib.lbm_kernel_launches(self._ctx)

    @property
    def storage_scale(self) -> float:
        return self._lib.lbm_storage_scale(self._ctx)

    def set_kernel(self, kernel):
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        self._check(self._lib.lbm_set_kernel(self._ctx, k))

    @property
    def kernel(self) -> str:
        k = self._lib.lbm_get_kernel(self._ctx)
        return {v: n for n, v in KERNELS.items()}[k]

    def autotune(self, trial_steps: int = 20):
        """Pick the fastest kernel / staged shape for this lattice by timing
        (state preserved); returns (kernel name, us per step)."""
        k, us = ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.lbm_autotune(self._ctx, int(trial_steps), ctypes.byref(k),
                                           ctypes.byref(us)))
        return {v: n for n, v in KERNELS.items()}[k.value], us.value

    def set_staged_config(self, stages: int = 0, ctas_per_sm: int = 0, consumer_warps: int = 0,
                          l2_evict_first: bool = False):
        """Shape of the staged kernel (0 = default); see lbm_set_staged_config."""
        self._check(self._lib.lbm_set_staged_config(self._ctx, int(stages), int(ctas_per_sm),
                                                    int(consumer_warps), int(l2_evict_first)))

    @property
    def staged_config(self):
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self._lib.lbm_get_staged_config(self._ctx, *[ctypes.byref(x) for x in v]))
        keys = ("stages", "ctas_per_sm", "consumer_warps", "l2_evict_first", "grid")
        return dict(zip(keys, (x.value for x in v)))

    def set_graph_chunk(self, steps: int):
        self._check(self._lib.lbm_set_graph_chunk(self._ctx, int(steps)))

    def set_wave_config(self, steps: int, rows: int):
        """Steps per launch and rows per segment of the multi-step kernel
        (lbm_set_wave_config)."""
        self._check(self._lib.lbm_set_wave_config(self._ctx, int(steps), int(rows)))

    @property
    def wave_config(self):
        v = [ctypes.c_int() for _ in range(2)]
        self._check(self._lib.lbm_get_wave_config(self._ctx, *[ctypes.byref(x) for x in v]))
        return {"steps": v[0].value, "rows": v[1].value}

    def set_launch_timing(self, on: bool):
        """Event pairs around every stream-collide launch (lbm_set_launch_timing)."""
        self._check(self._lib.lbm_set_launch_timing(self._ctx, int(bool(on))))

    def launch_time(self, which: int):
        """(milliseconds, launches, steps) of one kind of launch since timing
        was turned on (lbm_launch_time; TIMED_WAVE, TIMED_SINGLE or
        TIMED_RESIDUAL)."""
        ms, n, k = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self._lib.lbm_launch_time(self._ctx, int(which), ctypes.byref(ms),
                                              ctypes.byref(n), ctypes.byref(k)))
        return ms.value, n.value, k.value

    @property
    def bytes_per_site_update(self) -> float:
        """Algorithmic bytes per site update: one state buffer read and one
        written per node, i.e. 8 populations each way and, with 16-bit
        storage, the node's share of its tile's references."""
        nbytes = self._lib.lbm_population_bytes(Grid(self.nx, self.ny), self.precision)
        return 2.0 * nbytes / (self.nx * self.ny)


def _instances(instances):
    """ctypes array of lbm_instance from dicts (nx, ny, tau_N, tau_R and
    optional bc_x, bc_y, delta_e)."""
    arr = (Instance * len(instances))()
    for a, i in zip(arr, instances):
        a.nx, a.ny = int(i["nx"]), int(i["ny"])
        a.tau_N, a.tau_R = float(i["tau_N"]), float(i["tau_R"])
        a.bc = Boundary(int(i.get("bc_x", PERIODIC)), int(i.get("bc_y", PERIODIC)),
                        float(i.get("delta_e", 0.0)))
    return arr


def analytic_profiles(instances, out=None, op=0):
    """lbm_analytic_profiles: the Eq. 68 start of each instance in the
    layout of Batch.profiles(); op 0 returns them (a new CUDA float32
    tensor [n, 512]), op 1 / -1 adds them to / subtracts them from `out`
    in place."""
    import torch
    lib = load_library()
    if out is None:
        out = torch.empty((len(instances), 512), dtype=torch.float32, device="cuda")
    assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
    assert out.shape == (len(instances), 512)
    st = lib.lbm_analytic_profiles(_instances(instances), len(instances),
                                   ctypes.c_void_p(out.data_ptr()), int(op),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != OK:
        raise LBMError(st, lib.lbm_last_error(None).decode())
    return out


class Batch:
    """Many independent lattices advanced by one launch per step (see the
    batched solver in include/phonon_lbm.h).  ``instances`` is a list of
    dicts with keys nx, ny, tau_N, tau_R and optional bc_x, bc_y, delta_e."""

    def __init__(self, instances, precision="fp32", e_ref=1.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the phonon LBM runs only on the GPU")
        self._lib = load_library()
        self.torch = torch
        self.instances = [dict(i) for i in instances]
        arr = _instances(self.instances)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.stream = torch.cuda.current_stream()
        self._b = ctypes.c_void_p()
        st = self._lib.lbm_batch_create(arr, len(instances), self.precision, float(e_ref),
                                        ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(self._b))
        if st != OK:
            self._b = ctypes.c_void_p()
            raise LBMError(st, self._lib.lbm_last_error(None).decode())

    def _check(self, st):
        if st != OK:
            raise LBMError(st, self._lib.lbm_batch_last_error(self._b).decode())

    def close(self):
        if self._b:
            self._lib.lbm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def count(self):
        return len(self.instances)

    def init(self, e=None, qx=None, qy=None):
        """Step 0 from per-instance host fields (lists of [ny, nx] arrays) or
        the cold start (e = e_ref, q = 0) when omitted."""
        def cat(fields):
            if fields is None:
                return None
            return np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64).ravel()
                                                        for f in fields]))
        e, qx, qy = cat(e), cat(qx), cat(qy)
        p = lambda a: _dptr(a) if a is not None else None
        self._check(self._lib.lbm_batch_init(self._b, p(e), p(qx), p(qy)))

    def step(self, n=1):
        self._check(self._lib.lbm_batch_step(self._b, int(n)))

    def residuals(self):
        r = np.empty(self.count)
        en = np.full(self.count, np.nan)
        self._check(self._lib.lbm_batch_residuals(self._b, _dptr(r), _dptr(en)))
        return r, en

    def solve(self, tol=1e-8, check_every=100, max_steps=10 ** 6):
        steps = (ctypes.c_long * self.count)()
        r = np.empty(self.count)
        self._check(self._lib.lbm_batch_solve(self._b, float(tol), int(check_every),
                                              int(max_steps), steps, _dptr(r)))
        return np.array(steps[:], dtype=np.int64), r

    def moments(self, i):
        nx, ny = self.instances[i]["nx"], self.instances[i]["ny"]
        e = np.empty((ny, nx))
        qx = np.empty_like(e)
        qy = np.empty_like(e)
        self._check(self._lib.lbm_batch_moments(self._b, int(i), _dptr(e), _dptr(qx), _dptr(qy)))
        return e, qx, qy

    def set_schedule(self, threads_per_item=256, ctas_per_sm=0):
        self._check(self._lib.lbm_batch_set_schedule(self._b, int(threads_per_item),
                                                     int(ctas_per_sm)))

    @property
    def schedule(self):
        v = [ctypes.c_int() for _ in range(3)]
        self._check(self._lib.lbm_batch_get_schedule(self._b, *[ctypes.byref(x) for x in v]))
        return dict(zip(("threads_per_item", "ctas_per_sm", "grid"), (x.value for x in v)))

    def autotune(self, trial_steps=10):
        us = ctypes.c_double()
        self._check(self._lib.lbm_batch_autotune(self._b, int(trial_steps), ctypes.byref(us)))
        return us.value

    def set_wave(self, steps, rows=128):
        """Multi-step launches (lbm_batch_set_wave; steps 0 = one step per launch)."""
        self._check(self._lib.lbm_batch_set_wave(self._b, int(steps), int(rows)))

    @property
    def wave(self):
        v = [ctypes.c_int() for _ in range(2)]
        self._check(self._lib.lbm_batch_get_wave(self._b, *[ctypes.byref(x) for x in v]))
        return {"steps": v[0].value, "rows": v[1].value}

    def profiles(self):
        """Normalised steady profiles [count, 512] (CUDA float32 tensor)."""
        out = self.torch.empty((self.count, 512), dtype=self.torch.float32, device="cuda")
        self._check(self._lib.lbm_batch_profiles(self._b, ctypes.c_void_p(out.data_ptr())))
        return out

    def init_profiles(self, profiles):
        """Step 0 from predicted profiles [count, 512] (CUDA float32)."""
        p = profiles.to(device="cuda", dtype=self.torch.float32).contiguous()
        assert p.shape == (self.count, 512)
        self._check(self._lib.lbm_batch_init_profiles(self._b, ctypes.c_void_p(p.data_ptr())))

    @property
    def active(self):
        return self._lib.lbm_batch_active(self._b)

    def steps_of(self, i):
        return self._lib.lbm_batch_steps(self._b, int(i))


class Mlp:
    """The warm-start network (see lbm_mlp_* in include/phonon_lbm.h)."""

    def __init__(self, widths, max_batch=4096):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the network runs only on the GPU")
        self._lib = load_library()
        self.torch = torch
        self.widths = [int(w) for w in widths]
        arr = (ctypes.c_int * len(self.widths))(*self.widths)
        self.stream = torch.cuda.current_stream()
        self._m = ctypes.c_void_p()
        st = self._lib.lbm_mlp_create(arr, len(self.widths), int(max_batch),
                                      ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(self._m))
        if st != OK:
            self._m = ctypes.c_void_p()
            raise LBMError(st, self._lib.lbm_last_error(None).decode())
        self.max_batch = int(max_batch)

    def _check(self, st):
        if st != OK:
            raise LBMError(st, self._lib.lbm_mlp_last_error(self._m).decode())

    def close(self):
        if self._m:
            self._lib.lbm_mlp_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self):
        return self._lib.lbm_mlp_param_count(self._m)

    def init_params(self, seed=0):
        """Seeded uniform(-a, a) weights, a = sqrt(6 / (fan_in + fan_out)),
        zero biases."""
        rng = np.random.default_rng(seed)
        parts = []
        for k, n in zip(self.widths[:-1], self.widths[1:]):
            a = np.sqrt(6.0 / (k + n))
            parts += [rng.uniform(-a, a, n * k), np.zeros(n)]
        self.set_params(np.concatenate(parts).astype(np.float32))

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.param_count
        self._check(self._lib.lbm_mlp_set_params(self._m, p.ctypes.data_as(ctypes.c_void_p)))

    def params(self):
        p = np.empty(self.param_count, dtype=np.float32)
        self._check(self._lib.lbm_mlp_get_params(self._m, p.ctypes.data_as(ctypes.c_void_p)))
        return p

    def _dev(self, a):
        t = self.torch.as_tensor(a, dtype=self.torch.float32, device="cuda")
        return t.contiguous()

    def forward(self, x):
        x = self._dev(x)
        y = self.torch.empty((x.shape[0], self.widths[-1]), dtype=self.torch.float32,
                             device="cuda")
        self._check(self._lib.lbm_mlp_forward(self._m, ctypes.c_void_p(x.data_ptr()),
                                              x.shape[0], ctypes.c_void_p(y.data_ptr())))
        return y

    def loss_grad(self, x, t):
        x, t = self._dev(x), self._dev(t)
        g = np.empty(self.param_count, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.lbm_mlp_loss_grad(self._m, ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                                ctypes.byref(loss),
                                                g.ctypes.data_as(ctypes.c_void_p)))
        return loss.value, g

    def train_step(self, x, t, lr):
        x, t = self._dev(x), self._dev(t)
        loss = ctypes.c_double()
        self._check(self._lib.lbm_mlp_train_step(self._m, ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                                 ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value

    def train(self, x, t, steps, batch, lr, lr_final, seed=0):
        """lbm_mlp_train: `steps` Adam steps on minibatches of the rows of
        (x, t) drawn on the device, one captured step replayed; returns the
        per-step losses (numpy float32)."""
        x, t = self._dev(x), self._dev(t)
        hist = np.empty(int(steps), dtype=np.float32)
        self._check(self._lib.lbm_mlp_train(
            self._m, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), x.shape[0],
            int(batch), int(steps), ctypes.c_float(lr), ctypes.c_float(lr_final),
            ctypes.c_ulonglong(seed), hist.ctypes.data_as(ctypes.c_void_p)))
        return hist


class LatticeND:
    """A periodic D1Q2 or D3Q14 lattice on one GPU (lbm_nd_*).

    ``shape`` is (nz, ny, nx) for D3Q14 and (nx,) for D1Q2; fields are numpy
    float64 arrays of that shape, fluxes carry a leading axis of the
    lattice's dimension (x, y, z).  ``precision`` is "fp32" or "fp64".
    """

    def __init__(self, lattice, shape, tau_N, tau_R, precision="fp32", e_ref=1.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the phonon LBM runs only on the GPU")
        self._lib = load_library()
        self.lattice = int(lattice)
        self.shape = tuple(int(v) for v in shape)
        self.dim = 3 if self.lattice == D3Q14 else 1
        if len(self.shape) != self.dim:
            raise ValueError("shape must have one entry per lattice dimension")
        nz, ny, nx = (self.shape if self.dim == 3 else (1, 1, self.shape[0]))
        self.Q = 14 if self.lattice == D3Q14 else 2
        self.n = nx * ny * nz
        self.stream = torch.cuda.current_stream()
        self._ctx = ctypes.c_void_p()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        st = self._lib.lbm_nd_create(self.lattice, nx, ny, nz, float(tau_N), float(tau_R), prec,
                                     float(e_ref), ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(self._ctx))
        if st != OK:
            self._ctx = ctypes.c_void_p()
            raise LBMError(st, self._lib.lbm_nd_last_error(None).decode())

    def _check(self, st):
        if st != OK:
            raise LBMError(st, self._lib.lbm_nd_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            self._lib.lbm_nd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def lattice_speed(lattice) -> float:
        """c / v_g of the lattice (lbm_nd_lattice_speed)."""
        return load_library().lbm_nd_lattice_speed(int(lattice))

    def init(self, e, q=None):
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(e, dtype=np.float64), self.shape))
        qa = None if q is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(q, dtype=np.float64), (self.dim,) + self.shape))
        self._check(self._lib.lbm_nd_init(self._ctx, _dptr(e),
                                          _dptr(qa) if qa is not None else None))

    def step(self, n=1):
        self._check(self._lib.lbm_nd_step(self._ctx, int(n)))

    def sync(self):
        self._check(self._lib.lbm_nd_sync(self._ctx))

    def moments(self):
        """(e [shape], q [dim, *shape]) of the current state."""
        e = np.empty(self.shape)
        q = np.empty((self.dim,) + self.shape)
        self._check(self._lib.lbm_nd_moments(self._ctx, _dptr(e), _dptr(q)))
        return e, q

    def populations(self):
        f = np.empty((self.Q,) + self.shape)
        self._check(self._lib.lbm_nd_populations(self._ctx, _dptr(f)))
        return f

    def energy(self) -> float:
        v = ctypes.c_double()
        self._check(self._lib.lbm_nd_energy(self._ctx, ctypes.byref(v)))
        return v.value

    @property
    def step_count(self) -> int:
        return self._lib.lbm_nd_step_count(self._ctx)
