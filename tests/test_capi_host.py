"""The C-ABI library loads and exports every declared symbol; host-side
argument checks (no GPU needed: lbm_create validates before touching CUDA)."""
import ctypes
import math
import os
import re

import pytest

import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return plbm.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "phonon_lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(plbm.EXPORTS) == names


def test_tau_from_kn_and_sizes(lib):
    assert plbm.tau_from_kn(0.01, 31.0) == pytest.approx(0.01 * 31 * math.sqrt(0.6), rel=1e-15)
    g = plbm.Grid(128, 32)
    assert lib.lbm_population_bytes(g, plbm.FP32) == 8 * 128 * 32 * 4
    # 16-bit storage: 8 planes, then 8 reference values per tile of 8 nodes
    # (nx a multiple of 8) or of one node
    assert lib.lbm_population_bytes(g, plbm.FP16_DEV) == (8 * 128 * 32 + 8 * 16 * 32) * 2
    assert lib.lbm_population_bytes(g, plbm.BF16_DEV) == (8 * 128 * 32 + 8 * 16 * 32) * 2
    assert lib.lbm_population_bytes(plbm.Grid(37, 29), plbm.FP16_DEV) == 16 * 37 * 29 * 2
    assert lib.lbm_population_bytes(g, plbm.FP64) == 8 * 128 * 32 * 8
    assert lib.lbm_population_bytes(plbm.Grid(0, 3), plbm.FP32) == 0
    assert lib.lbm_population_bytes(g, 9) == 0


def _create(lib, nx=8, ny=8, tau_N=1.0, tau_R=2.0, bcx=0, bcy=0, de=0.0, prec=0, e_ref=1.0):
    ctx = ctypes.c_void_p()
    st = lib.lbm_create(plbm.Grid(nx, ny), tau_N, tau_R, plbm.Boundary(bcx, bcy, de), prec,
                        e_ref, None, ctypes.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("kw,status", [
    (dict(nx=0), plbm.EINVAL),
    (dict(ny=-1), plbm.EINVAL),
    (dict(tau_N=0.0), plbm.EINVAL),
    (dict(tau_R=-1.0), plbm.EINVAL),
    (dict(tau_N=float("nan")), plbm.EINVAL),
    (dict(tau_N=math.inf, tau_R=math.inf), plbm.EINVAL),
    (dict(bcx=plbm.DIFFUSE_WALLS), plbm.EUNSUPPORTED),
    (dict(bcy=plbm.PERIODIC_GRADIENT), plbm.EUNSUPPORTED),
    (dict(bcx=7), plbm.EINVAL),
    (dict(bcy=plbm.DIFFUSE_WALLS, ny=1), plbm.EINVAL),
    (dict(de=math.inf, bcx=1), plbm.EINVAL),
    (dict(e_ref=math.nan), plbm.EINVAL),
    (dict(prec=4), plbm.EINVAL),
])
def test_create_rejects_bad_arguments(lib, kw, status):
    st, ctx = _create(lib, **kw)
    assert st == status
    assert not ctx.value
    assert lib.lbm_last_error(None)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == plbm.EINVAL
    assert lib.lbm_residual(None, None, None) == plbm.EINVAL
    assert lib.lbm_moments(None, None, None, None) == plbm.EINVAL
    assert lib.lbm_step_count(None) == -1
    assert lib.lbm_state_bytes(None) == 0
    lib.lbm_destroy(None)
    st = lib.lbm_create_ex(plbm.Grid(4, 4), 1.0, 1.0, plbm.Boundary(0, 0, 0.0), 0, 1.0, None,
                           None, None, 0, ctypes.byref(ctypes.c_void_p()))
    assert st == plbm.EINVAL
