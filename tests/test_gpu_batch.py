"""Batched solver: many instances advanced by one launch per step."""
import math

import numpy as np
import pytest

import oracle
import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs
from tests.helpers import TOL, check_gate, err_metrics, oracle_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

G, W = plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS

# uneven sizes, boundaries and relaxation times (nx multiple of 8)
MIXED = [
    dict(nx=64, ny=16, tau_N=0.9, tau_R=12.0, bc_x=G, bc_y=W, delta_e=1e-3),
    dict(nx=256, ny=40, tau_N=1.7, tau_R=3.0, bc_x=plbm.PERIODIC, bc_y=plbm.PERIODIC),
    dict(nx=40, ny=33, tau_N=0.4, tau_R=math.inf, bc_x=G, bc_y=plbm.PERIODIC, delta_e=-2e-3),
    dict(nx=1024, ny=3, tau_N=5.0, tau_R=0.9, bc_x=G, bc_y=W, delta_e=5e-4),
    dict(nx=8, ny=2, tau_N=0.8, tau_R=7.0, bc_x=G, bc_y=W, delta_e=1e-3),
]


def _fields(inst, seed):
    return [inputs.random_state_fields(i["nx"], i["ny"], seed=seed + k)
            for k, i in enumerate(inst)]


@pytest.mark.parametrize("precision", ["fp32", "fp16", "fp64"])
@pytest.mark.parametrize("tpi", [128, 256, 512])
def test_batch_equals_single_lattices_bitwise(precision, tpi):
    fields = _fields(MIXED, 100)
    b = plbm.Batch(MIXED, precision=precision)
    b.set_schedule(tpi)
    b.init(*[list(x) for x in zip(*fields)])
    b.step(37)
    for k, i in enumerate(MIXED):
        lat = plbm.Lattice(i["nx"], i["ny"], i["tau_N"], i["tau_R"], i.get("bc_x", 0),
                           i.get("bc_y", 0), i.get("delta_e", 0.0), precision=precision,
                           kernel="vector")
        lat.init(*fields[k])
        if precision in ("fp16", "bf16"):
            # one storage scale for the whole batch: compare with the oracle
            o = oracle_run(i["nx"], i["ny"], i["tau_N"], i["tau_R"], fields[k], 37,
                           i.get("bc_x", 0), i.get("bc_y", 0), i.get("delta_e", 0.0))
            err_e, err_q = err_metrics(b.moments(k), o.moments())
            check_gate(precision, err_e, err_q)
            continue
        lat.step(37)
        for x, y in zip(b.moments(k), lat.moments()):
            assert np.array_equal(x, y), k


def test_batch_matches_oracle():
    fields = _fields(MIXED, 7)
    b = plbm.Batch(MIXED)
    b.init(*[list(x) for x in zip(*fields)])
    b.step(60)
    for k, i in enumerate(MIXED):
        o = oracle_run(i["nx"], i["ny"], i["tau_N"], i["tau_R"], fields[k], 60,
                       i.get("bc_x", 0), i.get("bc_y", 0), i.get("delta_e", 0.0))
        err_e, err_q = err_metrics(b.moments(k), o.moments())
        assert err_e <= TOL["fp32"] and err_q <= TOL["fp32"], (k, err_e, err_q)


def test_batch_residuals_match_single_lattice():
    fields = _fields(MIXED[:2], 3)
    b = plbm.Batch(MIXED[:2])
    b.init(*[list(x) for x in zip(*fields)])
    lats = []
    for k, i in enumerate(MIXED[:2]):
        lat = plbm.Lattice(i["nx"], i["ny"], i["tau_N"], i["tau_R"], i.get("bc_x", 0),
                           i.get("bc_y", 0), i.get("delta_e", 0.0), kernel="vector")
        lat.init(*fields[k])
        lats.append(lat)
    for n in (5, 20):
        b.step(n)
        r, en = b.residuals()
        for k, lat in enumerate(lats):
            lat.step(n)
            if n == 5:
                lat.step(0)
            rl, el = lat.residual()
            if n == 5:
                assert math.isinf(r[k]) and math.isinf(rl)
            else:
                assert r[k] == pytest.approx(rl, rel=1e-12)
            assert en[k] == pytest.approx(el, rel=1e-13)


def _channels(n, seed, w_range):
    out = []
    for c in inputs.batch_channels(4 * n, seed=seed, w_range=w_range):
        tau_N = oracle.tau_from_kn(c["kn_N"], c["d"])
        tau_R = oracle.tau_from_kn(c["kn_R"], c["d"])
        if oracle.params(tau_N, tau_R)["tau"] < 0.6:      # linear-stability bound
            continue
        out.append(dict(nx=c["nx"], ny=c["ny"], tau_N=tau_N, tau_R=tau_R, bc_x=G, bc_y=W,
                        delta_e=1e-3, kn_N=c["kn_N"], kn_R=c["kn_R"]))
        if len(out) == n:
            break
    return out


def test_batch_solve_to_steady_state_and_retire():
    inst = _channels(12, seed=11, w_range=(16, 40))
    b = plbm.Batch(inst)
    b.init()                                   # cold start: e = e_ref, q = 0
    steps, r = b.solve(tol=1e-8, check_every=100, max_steps=200000)
    assert b.active == 0
    assert np.all(r < 1e-8), r
    assert len(set(steps.tolist())) > 1       # instances converge at different times
    # a retired instance's state equals a single lattice run for its steps
    for k in (0, len(inst) - 1):
        i = inst[k]
        lat = plbm.Lattice(i["nx"], i["ny"], i["tau_N"], i["tau_R"], G, W, 1e-3, kernel="vector")
        lat.init(np.ones((i["ny"], i["nx"])))
        lat.step(int(steps[k]))
        for x, y in zip(b.moments(k), lat.moments()):
            assert np.array_equal(x, y), k
        # and its core heat-flux profile is the phonon Poiseuille profile (Eq. 68)
        e, qx, _ = b.moments(k)
        slope = np.polyfit(np.arange(i["nx"]), e.mean(0), 1)[0]
        Q = qx.mean(1) / (-(5 / 9) * i["tau_R"] * slope)
        from tests.test_oracle_pins import eq68
        Y = np.arange(i["ny"]) / (i["ny"] - 1)
        core = (Y >= 0.2) & (Y <= 0.8)
        assert np.abs(Q - eq68(Y, i["kn_N"], i["kn_R"]))[core].max() < 0.05


def test_batch_autotune_keeps_state():
    fields = _fields(MIXED, 55)
    a = plbm.Batch(MIXED)
    a.init(*[list(x) for x in zip(*fields)])
    a.step(9)
    b = plbm.Batch(MIXED)
    b.init(*[list(x) for x in zip(*fields)])
    b.step(9)
    us = b.autotune(4)
    assert us > 0 and b.schedule["threads_per_item"] in (128, 256, 512)
    a.step(11)
    b.step(11)
    for k in range(len(MIXED)):
        for x, y in zip(a.moments(k), b.moments(k)):
            assert np.array_equal(x, y)


def test_batch_rejects_bad_instances():
    with pytest.raises(plbm.LBMError) as ex:
        plbm.Batch([dict(nx=30, ny=4, tau_N=1.0, tau_R=1.0)])
    assert ex.value.status == plbm.EINVAL and "instance 0" in str(ex.value)
    with pytest.raises(plbm.LBMError) as ex:
        plbm.Batch([MIXED[0], dict(nx=64, ny=4, tau_N=1.0, tau_R=1.0, bc_y=G)])
    assert ex.value.status == plbm.EUNSUPPORTED and "instance 1" in str(ex.value)


def test_full_512_channel_batch_in_bench_configuration():
    """The batched workload at its full size (512 seeded channels, 1.95e8
    sites) in the bench's launch configuration (autotuned schedule), from the
    cold start: the three smallest channels against the oracle element by
    element, three others bit-identical to single-lattice runs."""
    import bench
    inst, _ = bench.batch_instances(512)
    b = plbm.Batch(inst)
    b.init()
    b.autotune(4)
    b.init()
    steps = 24
    b.step(steps)
    sizes = np.array([i["nx"] * i["ny"] for i in inst])
    small = np.argsort(sizes)[:3].tolist()
    rng = np.random.default_rng(3)
    other = rng.choice([k for k in range(len(inst)) if k not in small], 3, replace=False)
    ones = lambda i: np.ones((i["ny"], i["nx"]))
    for k in small:
        i = inst[k]
        o = oracle_run(i["nx"], i["ny"], i["tau_N"], i["tau_R"], (ones(i), None, None), steps,
                       i["bc_x"], i["bc_y"], i["delta_e"])
        eo, qxo, qyo = o.moments()
        eg, qxg, qyg = b.moments(k)
        # cold start: e - 1 and q start at zero, so scale by the oracle's range
        err_e = np.abs(eg - eo).max() / max(np.abs(eo - 1.0).max(), 1e-30)
        err_q = max(np.abs(qxg - qxo).max(), np.abs(qyg - qyo).max()) / \
            max(np.abs(qxo).max(), np.abs(qyo).max())
        assert err_e <= TOL["fp32"] and err_q <= TOL["fp32"], (k, err_e, err_q)
    for k in other:
        i = inst[int(k)]
        lat = plbm.Lattice(i["nx"], i["ny"], i["tau_N"], i["tau_R"], i["bc_x"], i["bc_y"],
                           i["delta_e"], kernel="vector")
        lat.init(ones(i))
        lat.step(steps)
        for x, y in zip(b.moments(int(k)), lat.moments()):
            assert np.array_equal(x, y), k
        lat.close()
    b.close()


# --- multi-step launches (lbm_batch_set_wave) -------------------------------
WAVE_MIXED = [dict(i) for i in MIXED] + [
    dict(nx=132, ny=21, tau_N=0.9, tau_R=4.0, bc_x=G, bc_y=W, delta_e=1e-3)]   # ragged strips


@pytest.mark.parametrize("steps,rows", [(2, 7), (3, 64), (4, 128), (8, 5)])
def test_batch_wave_equals_single_steps_bitwise(steps, rows):
    """Multi-step launches of every instance (uneven sizes, both boundary
    kinds, strips that wrap and ragged last strips) give the single-step
    batch's states bit for bit, through steps, residuals and a solve."""
    fields = _fields(WAVE_MIXED, 17)
    args = [list(x) for x in zip(*fields)]
    a = plbm.Batch(WAVE_MIXED)
    a.init(*args)
    b = plbm.Batch(WAVE_MIXED)
    b.set_wave(steps, rows)
    assert b.wave == {"steps": steps, "rows": rows}
    b.init(*args)
    for n in (1, 2, 37):
        a.step(n)
        b.step(n)
        for k in range(len(WAVE_MIXED)):
            for x, y in zip(a.moments(k), b.moments(k)):
                assert np.array_equal(x, y), (n, k)
    ra, ea = a.residuals()
    rb, eb = b.residuals()
    assert np.array_equal(ea, eb)
    sa, ra = a.solve(tol=1e-3, check_every=26, max_steps=260)
    sb, rb = b.solve(tol=1e-3, check_every=26, max_steps=260)
    assert np.array_equal(sa, sb) and np.array_equal(ra, rb)
    for k in range(len(WAVE_MIXED)):
        for x, y in zip(a.moments(k), b.moments(k)):
            assert np.array_equal(x, y), ("solve", k)


def test_batch_wave_refusals():
    b = plbm.Batch(MIXED, precision="fp16")
    with pytest.raises(plbm.LBMError) as ex:
        b.set_wave(4)
    assert ex.value.status == plbm.EUNSUPPORTED
    c = plbm.Batch(MIXED)
    for steps, rows in ((1, 64), (9, 64), (4, 0)):
        with pytest.raises(plbm.LBMError) as ex:
            c.set_wave(steps, rows)
        assert ex.value.status == plbm.EINVAL
    c.set_wave(0)
    assert c.wave["steps"] == 0
