"""The multi-step kernel (LBM_KERNEL_WAVE): several time steps per launch,
bit-identical to single steps.  Its oracle parity runs in the parity sweep
of test_gpu_parity.py; here: every steps-per-launch and segment height
against the scalar kernel, the stepping plan (graphs, remainders, the
closing single step, lbm_step_residual), checkpoints, launch timing,
refusals, and the 8192^2 bench configuration against the vector kernel."""
import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs
from tests.helpers import check_gate, err_metrics, oracle_run, tau_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

GRAD, WALLS, PER = plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, plbm.PERIODIC

# (nx, ny, bc_x, bc_y): strips that wrap (nx < 64), ragged last strips,
# two wall rows only, periodic rows fewer than the steps per launch
CASES = [(256, 64, GRAD, WALLS), (130, 50, PER, PER), (64, 9, GRAD, WALLS), (2, 3, GRAD, PER),
         (1000, 37, GRAD, WALLS), (6, 2, GRAD, WALLS), (118, 5, GRAD, PER)]


def lattice(nx, ny, bx, by, kernel, **kw):
    return plbm.Lattice(nx, ny, 0.9, 12.0, bx, by, 1e-3, kernel=kernel, **kw)


def fields(nx, ny):
    return inputs.random_state_fields(nx, ny, seed=7 * nx + ny)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_bc{c[2]}{c[3]}")
def test_every_shape_bit_identical_to_single_steps(case):
    nx, ny, bx, by = case
    f = fields(nx, ny)
    ref = lattice(nx, ny, bx, by, "scalar")
    ref.init(*f)
    ref.step(37)
    want = ref.populations()
    # the residual step of a wave lattice runs on the vector kernel when nx
    # allows (its block sums, hence the last bits of the totals, follow it)
    single = "vector" if nx % 4 == 0 else "scalar"
    rs = lattice(nx, ny, bx, by, single)
    rs.init(*f)
    rs.step(37)
    want_r = rs.step_residual(9)
    for K in range(2, 9):
        for rows in (1, 5, 64):
            g = lattice(nx, ny, bx, by, "wave")
            g.set_wave_config(K, rows)
            g.init(*f)
            g.step(37)
            assert g.step_count == 37
            assert np.array_equal(g.populations(), want), (K, rows)
            assert g.step_residual(9) == want_r, (K, rows)
            g.close()


def test_stepping_plan_graphs_and_remainders():
    """Mixed lbm_step / lbm_step_residual calls, with and without graphs,
    every remainder of the steps per launch: same bits as single steps."""
    nx, ny = 192, 70
    f = fields(nx, ny)
    calls = [1, 2, 3, 7, ("r", 1), ("r", 2), 130, ("r", 100), 64, 5, ("r", 13), 200]
    ref = lattice(nx, ny, GRAD, WALLS, "vector")
    ref.init(*f)
    outs = []
    for c in calls:
        if isinstance(c, tuple):
            outs.append(ref.step_residual(c[1]))
        else:
            ref.step(c)
        outs.append(ref.populations())
    for K, chunk in ((4, 64), (5, 0), (3, 16), (8, 64)):
        g = lattice(nx, ny, GRAD, WALLS, "wave", graph_chunk=chunk)
        g.set_wave_config(K, 32)
        g.init(*f)
        got = []
        for c in calls:
            if isinstance(c, tuple):
                got.append(g.step_residual(c[1]))
            else:
                g.step(c)
            got.append(g.populations())
        assert g.step_count == ref.step_count
        for a, b in zip(outs, got):
            if isinstance(a, tuple):
                assert a == b, (K, chunk)
            else:
                assert np.array_equal(a, b), (K, chunk)


def test_checkpoint_resume():
    nx, ny = 256, 40
    f = fields(nx, ny)
    g = lattice(nx, ny, GRAD, WALLS, "wave")
    g.init(*f)
    g.step(45)
    blob = g.get_state()
    g.step(80)
    h = lattice(nx, ny, GRAD, WALLS, "wave")
    h.set_state(blob)
    assert h.step_count == 45
    h.step(80)
    assert np.array_equal(g.populations(), h.populations())


def test_launch_timing_counts():
    nx, ny = 512, 128
    g = lattice(nx, ny, GRAD, WALLS, "wave")
    g.set_wave_config(4, 64)
    g.init(*fields(nx, ny))
    g.set_launch_timing(True)
    g.step_residual(100)        # 99 plain steps: 24 launches of 4, one of 3
    g.step(10)                  # 9 steps in launches of 4, then 2 single steps
    ms, n, k = g.launch_time(plbm.TIMED_WAVE)
    assert (n, k) == (24 + 1 + 2, 99 + 8) and ms > 0
    assert g.launch_time(plbm.TIMED_RESIDUAL)[1:] == (1, 1)
    assert g.launch_time(plbm.TIMED_SINGLE)[1:] == (2, 2)
    g.set_launch_timing(False)
    assert g.launch_time(plbm.TIMED_WAVE) == (0.0, 0, 0)


# 16-bit storage: levels in FP32 between launches, so a launch is not the
# bits of single 16-bit steps; checked against the oracle (the 16-bit gate)
CASES16 = [(256, 64, GRAD, WALLS), (128, 50, PER, PER), (64, 9, GRAD, WALLS),
           (8, 5, GRAD, PER), (120, 6, GRAD, WALLS), (16, 2, GRAD, WALLS)]


@pytest.mark.parametrize("precision,rounding", [("fp16", "nearest"), ("fp16", "stochastic"),
                                                ("bf16", "nearest"), ("bf16", "stochastic")])
@pytest.mark.parametrize("case", CASES16, ids=lambda c: f"{c[0]}x{c[1]}_bc{c[2]}{c[3]}")
def test_16bit_multi_step_against_oracle(case, precision, rounding):
    nx, ny, bx, by = case
    f = fields(nx, ny)
    steps = 37
    o = oracle_run(nx, ny, 0.9, 12.0, f, steps, bx, by, 1e-3)
    ref = o.moments()

    def run(prec, kernel, K=4, rows=64):
        g = lattice(nx, ny, bx, by, kernel, precision=prec, rounding=rounding)
        if kernel == "wave":
            g.set_wave_config(K, rows)
        g.init(*f)
        g.step(steps)
        m = g.moments()
        g.close()
        return m

    single = max(err_metrics(run(precision, "vector"), ref))
    worst = None
    for K, rows in ((2, 7), (3, 64), (4, 1), (4, 64)):
        m = run(precision, "wave", K, rows)
        assert np.array_equal(m[0], run(precision, "wave", K, rows)[0])     # deterministic
        err = err_metrics(m, ref)
        # one rounding per launch instead of per step: no worse than single steps
        assert max(err) <= 1.5 * single + 1e-6, (K, rows, err, single)
        if worst is None or max(err) > max(worst[0]):
            worst = (err, K, rows)
    (err_e, err_q), K, rows = worst
    check_gate(precision, err_e, err_q,
               fp16=lambda: err_metrics(run("fp16", "wave", K, rows), ref))


def test_refusals():
    with pytest.raises(plbm.LBMError) as ex:
        plbm.Lattice(252, 16, 0.9, 12.0, GRAD, WALLS, 1e-3, precision="fp16", kernel="wave")
    assert ex.value.status == plbm.EUNSUPPORTED          # 16-bit: nx a multiple of 8
    with pytest.raises(plbm.LBMError) as ex:
        plbm.Lattice(256, 16, 0.9, 12.0, GRAD, WALLS, 1e-3, precision="fp64", kernel="wave")
    assert ex.value.status == plbm.EUNSUPPORTED
    h = plbm.Lattice(256, 16, 0.9, 12.0, GRAD, WALLS, 1e-3, precision="bf16", kernel="wave")
    with pytest.raises(plbm.LBMError) as ex:
        h.set_wave_config(5, 64)                          # 16-bit: up to 4 steps
    assert ex.value.status == plbm.EINVAL
    with pytest.raises(plbm.LBMError) as ex:
        plbm.Lattice(255, 16, 0.9, 12.0, GRAD, WALLS, 1e-3, kernel="wave")      # nx odd
    assert ex.value.status == plbm.EUNSUPPORTED
    with pytest.raises(plbm.LBMError) as ex:
        plbm.Lattice(256, 16, 0.9, 12.0, plbm.SIDES, WALLS, 0.0, kernel="wave")
    assert ex.value.status == plbm.EUNSUPPORTED
    g = lattice(256, 16, GRAD, WALLS, "wave")
    for K, rows in ((1, 64), (9, 64), (4, 0)):
        with pytest.raises(plbm.LBMError) as ex:
            g.set_wave_config(K, rows)
        assert ex.value.status == plbm.EINVAL
    assert g.wave_config == {"steps": 4, "rows": 128}


def test_8192_bench_configuration_bit_identical_to_vector_kernel():
    """The bench workload at full size in the bench's launch configuration
    (autotuned; the multi-step kernel with each shape the autotuner tries):
    after 300 steps, with residual windows, every node's moments equal the
    vector kernel's bit for bit (the vector kernel is checked against the
    oracle on light-cone windows of the same workload)."""
    w = inputs.THROUGHPUT_8192
    tau_N, tau_R = tau_pair(w.kn_N, w.kn_R, w.length)
    e, qx, qy = inputs.initial_fields(w)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (e, qx, qy)]

    def run(kernel, shape=None, tune=False):
        g = plbm.Lattice(w.nx, w.ny, tau_N, tau_R, kernel=kernel)
        g.init(*t)
        if tune:
            g.autotune(20)
        if shape:
            g.set_wave_config(*shape)
        g.step_residual(100)
        g.step(199)
        m = [x.clone() for x in g.moments_device()]
        info = (g.kernel, g.wave_config)
        g.close()
        return m, info

    want, _ = run("vector")
    got, info = run("auto", tune=True)
    for a, b in zip(want, got):
        assert torch.equal(a, b), info
    for shape in ((4, 64), (6, 128)):
        got, _ = run("wave", shape)
        for a, b in zip(want, got):
            assert torch.equal(a, b), shape


@pytest.mark.parametrize("precision,rounding", [("fp16", "nearest"), ("bf16", "stochastic")])
def test_16bit_multi_step_graphs_and_checkpoints_agree(precision, rounding):
    """16-bit multi-step launches: captured graphs, direct launches and a
    checkpoint round trip store the same bits (the same launches in the same
    order), through residual windows."""
    nx, ny = 256, 72
    f = fields(nx, ny)
    outs = []
    for chunk in (64, 0, 16):
        g = lattice(nx, ny, GRAD, WALLS, "wave", precision=precision, rounding=rounding,
                    graph_chunk=chunk)
        g.init(*f)
        g.step(130)
        r = g.step_residual(50)
        g.step(7)
        outs.append((g.populations(), r))
        g.close()
    for p, r in outs[1:]:
        assert np.array_equal(p, outs[0][0]) and r == outs[0][1]
    g = lattice(nx, ny, GRAD, WALLS, "wave", precision=precision, rounding=rounding)
    g.init(*f)
    g.step(130)
    blob = g.get_state()
    g.step_residual(50)
    g.step(7)
    h = lattice(nx, ny, GRAD, WALLS, "wave", precision=precision, rounding=rounding)
    h.set_state(blob)
    h.step_residual(50)
    h.step(7)
    assert np.array_equal(g.populations(), h.populations())
