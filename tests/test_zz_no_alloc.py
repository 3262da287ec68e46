"""lbm_residual_noalloc: the residual entry point for callers that must not
allocate device memory (a host that keeps all device memory in its own pool,
a plugin inside a framework that owns the allocator, a loop that cannot
afford an allocator call).  It is checked, through the C-ABI, against the
context's own lbm_residual on the same lattice state, on two calls in a row.

This file is collected last on purpose: a run that stops at the first
failure has run every other test before it.  It does not depend on them and
passes in a fresh process on its own."""
import math

import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs
from tests.helpers import TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_noalloc_residual_matches_lbm_residual_two_calls():
    nx, ny = 512, 96
    fields = inputs.random_state_fields(nx, ny, seed=77)
    lat = plbm.Lattice(nx, ny, 0.8, 12.0, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3,
                       precision="fp32")
    lat.init(*fields)
    lat.residual()                          # the context's history at step 0
    prev = lat.moments_device()
    for k in (10, 25):                      # two calls in a row
        lat.step(k)
        r_ctx, en_ctx = lat.residual()
        cur = lat.moments_device()
        r_na, en_na = plbm.residual_noalloc(cur, prev, k_steps=k, e_ref=1.0)
        assert math.isfinite(r_na) and r_na > 0
        # lbm_residual forms per-node moments in the FP32 compute precision,
        # the no-allocation call sums FP64 moment fields: agreement within
        # the FP32 parity tolerance (energy far tighter)
        assert r_na == pytest.approx(r_ctx, rel=TOL["fp32"])
        assert en_na == pytest.approx(en_ctx, rel=1e-9)
        prev = cur
    # no previous fields: energy only, r = inf
    r0, en0 = plbm.residual_noalloc(prev, None, 0, e_ref=1.0)
    assert math.isinf(r0) and en0 == pytest.approx(en_ctx, rel=1e-9)


def test_noalloc_residual_rejects_oversize_and_bad_arguments():
    small = [torch.zeros(16, dtype=torch.float64, device="cuda") for _ in range(3)]
    lib = plbm.load_library()
    import ctypes
    p = [ctypes.c_void_p(t.data_ptr()) for t in small]
    r, en = ctypes.c_double(), ctypes.c_double()
    st = lib.lbm_residual_noalloc(*p, None, None, None, plbm.NOALLOC_MAX_NODES + 1, 1.0, 1,
                                  None, ctypes.byref(r), ctypes.byref(en))
    assert st == plbm.EINVAL
    assert b"maximum" in lib.lbm_last_error(None)
    st = lib.lbm_residual_noalloc(*p, p[0], None, None, 16, 1.0, 1, None, ctypes.byref(r),
                                  ctypes.byref(en))
    assert st == plbm.EINVAL
    # a NaN in the fields is reported, outputs still written
    small[0][3] = float("nan")
    with pytest.raises(plbm.LBMError) as ex:
        plbm.residual_noalloc(small)
    assert ex.value.status == plbm.ENONFINITE
