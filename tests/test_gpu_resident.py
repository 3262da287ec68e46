"""The cluster-resident kernel (LBM_KERNEL_RESIDENT: a small FP32 lattice
held in the shared memory of one thread-block cluster, n steps per launch)
against the scalar kernel bit for bit, and against the FP64 oracle on the
paper's grids."""
import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs
from tests.helpers import TOL, err_metrics, oracle_run, tau_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

S = plbm.SIDES
DIF, ISO, FLX = plbm.DIFFUSE, plbm.ISOTHERMAL, plbm.HEAT_FLUX

# (nx, ny, bc_x, bc_y, delta_e, sides): slabs of columns and of rows, one
# CTA and up to 16, ragged last slabs, every boundary kind
CASES = [
    (128, 32, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, None),   # the channel
    (4096, 4, plbm.PERIODIC, plbm.PERIODIC, 0.0, None),                  # second sound
    (3, 301, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, None),    # rows, one CTA
    (17, 1000, plbm.PERIODIC, plbm.DIFFUSE_WALLS, 0.0, None),            # 9 slabs of rows
    (201, 201, S, S, 0.0, [(ISO, 1.0), (ISO, 1.0), (ISO, 1.0), (FLX, 1e-4)]),  # 16 CTAs
    (401, 3, S, plbm.PERIODIC, 0.0, [(FLX, 1e-4), (DIF, 0.0), None, None]),
    (37, 29, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, -1e-3, None),
    (1, 1, plbm.PERIODIC, plbm.PERIODIC, 0.0, None),
    (2, 2, S, S, 0.0, [(ISO, 1.001), (ISO, 1.0), (DIF, 0.0), (FLX, 1e-4)]),
]


def _lattice(case, kernel, **kw):
    nx, ny, bcx, bcy, de, sides = case
    sides = {i: s for i, s in enumerate(sides or []) if s is not None}
    return plbm.Lattice(nx, ny, 0.9, 15.0, bcx, bcy, de, kernel=kernel, sides=sides, **kw)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_bc{c[2]}{c[3]}")
def test_resident_equals_scalar_bitwise(case):
    """Same populations, moments and residuals as the scalar kernel, whether
    the steps come as one launch, odd and even pieces, or single steps, and
    through a residual step in between (that one runs on the vector or
    scalar kernel)."""
    nx, ny = case[0], case[1]
    fields = inputs.random_state_fields(nx, ny, seed=nx * 7 + ny)
    out = []
    for kernel in ("scalar", "resident"):
        lat = _lattice(case, kernel)
        assert lat.kernel == kernel
        lat.init(*fields)
        lat.step(37)
        f37 = lat.populations()
        lat.step(1)
        lat.step(1)
        lat.step(4)
        lat.step_residual(10)               # sets the residual history
        r, en = lat.step_residual(10)
        lat.step(41)
        out.append((f37, lat.populations(), lat.moments(), r, en, lat.step_count))
    (a37, af, am, ar, ae, an), (b37, bf, bm, br, be, bn) = out
    assert an == bn == 104
    assert np.array_equal(a37, b37)
    assert np.array_equal(af, bf)
    for x, y in zip(am, bm):
        assert np.array_equal(x, y)
    # the residual step itself runs on the vector or scalar kernel, whose
    # sums group the nodes differently: equal to rounding
    assert ae == pytest.approx(be, rel=1e-12)
    assert (ar == br) if not np.isfinite(ar) else ar == pytest.approx(br, rel=1e-6)


def test_resident_one_launch_per_call_and_checkpoint():
    case = CASES[0]
    fields = inputs.random_state_fields(128, 32, seed=3)
    lat = _lattice(case, "resident")
    lat.init(*fields)
    before = lat.kernel_launches
    lat.step(1000)
    assert lat.kernel_launches - before == 1
    blob = lat.get_state()
    lat.step(333)
    ref = lat.populations()
    lat.set_state(blob)
    assert lat.step_count == 1000
    lat.step(333)
    assert np.array_equal(lat.populations(), ref)


def test_resident_refuses_what_it_cannot_hold():
    for precision in ("fp64", "fp16", "bf16"):
        lat = plbm.Lattice(128, 32, 0.9, 15.0, precision=precision)
        with pytest.raises(plbm.LBMError) as ei:
            lat.set_kernel("resident")
        assert ei.value.status == plbm.EUNSUPPORTED
    big = plbm.Lattice(1024, 1024, 0.9, 15.0)          # 64 MB of populations
    with pytest.raises(plbm.LBMError) as ei:
        big.set_kernel("resident")
    assert ei.value.status == plbm.EUNSUPPORTED
    assert big.kernel == "vector"


@pytest.mark.parametrize("kn_R", [0.1, 1.0, 10.0])
def test_resident_second_sound_4096x4_full(kn_R):
    """The 4096 x 4 second-sound pulse, 5000 steps in one launch, against the
    oracle within the FP32 gate."""
    w = inputs.second_sound_4096x4(kn_R)
    tau_N, tau_R = tau_pair(w.kn_N, w.kn_R, w.length)
    fields = inputs.initial_fields(w)
    g = plbm.Lattice(w.nx, w.ny, tau_N, tau_R, kernel="resident")
    g.init(*fields)
    g.step(w.steps)
    o = oracle_run(w.nx, w.ny, tau_N, tau_R, fields, w.steps)
    err_e, err_q = err_metrics(g.moments(), o.moments())
    assert err_e <= TOL["fp32"] and err_q <= TOL["fp32"], (err_e, err_q)


def test_resident_poiseuille_128x32_full():
    w = inputs.POISEUILLE_128x32
    tau_N, tau_R = tau_pair(w.kn_N, w.kn_R, w.length)
    fields = inputs.initial_fields(w)
    g = plbm.Lattice(w.nx, w.ny, tau_N, tau_R, w.bc_x, w.bc_y, w.delta_e, kernel="resident")
    g.init(*fields)
    g.step(w.steps)
    o = oracle_run(w.nx, w.ny, tau_N, tau_R, fields, w.steps, w.bc_x, w.bc_y, w.delta_e)
    err_e, err_q = err_metrics(g.moments(), o.moments())
    assert err_e <= TOL["fp32"] and err_q <= TOL["fp32"], (err_e, err_q)
