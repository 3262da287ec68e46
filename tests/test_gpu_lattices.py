"""GPU path of the D1Q2 / D3Q14 lattices (lbm_nd_*) against the FP64 oracle
``oracle/lattices.py`` on the same seeded inputs, element by element, and
against the exact Fourier-mode map on larger lattices."""
import math

import numpy as np
import pytest

from oracle import lattices as lt
import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs
from tests.helpers import TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

KIND = {"D3Q14": (plbm.D3Q14, lt.D3Q14), "D1Q2": (plbm.D1Q2, lt.D1Q2)}


def _fields(L, shape, seed):
    n = int(np.prod(shape))
    e = 1 + inputs.uniform_noise(shape, 1e-3, seed)
    q = np.stack([inputs.uniform_noise(shape, 1e-3, seed, (a + 1) << 40) for a in range(L.dim)])
    return e, q


def _errs(gpu, orc, scale_e, scale_q):
    """Largest errors of e and q relative to the size of the input's
    deviations (small lattices relax to uniform within the run, so the
    current spread is no scale)."""
    (eg, qg), (eo, qo) = gpu, orc
    return np.abs(eg - eo).max() / scale_e, np.abs(qg - qo).max() / scale_q


CASES = [
    ("D3Q14", (16, 16, 16)),
    ("D3Q14", (13, 10, 24)),      # ragged: no size a multiple of a warp
    ("D3Q14", (3, 2, 5)),
    ("D3Q14", (1, 1, 1)),
    ("D1Q2", (1000,)),
    ("D1Q2", (7,)),
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}_{'x'.join(map(str, c[1]))}")
def test_nd_parity(case, precision):
    name, shape = case
    kind, L = KIND[name]
    tau_N, tau_R = 0.9, 12.0
    e, q = _fields(L, shape, seed=sum(shape) * 31 + len(shape))
    g = plbm.LatticeND(kind, shape, tau_N, tau_R, precision=precision)
    g.init(e, q)
    o = lt.Run(L, shape, tau_N, tau_R)
    o.init(e, q)
    tol = TOL[precision]
    scale_e, scale_q = np.abs(e - 1.0).max(), np.abs(q).max()
    scale_f = np.abs(o.f - L.w.reshape((L.Q,) + (1,) * L.dim)).max()
    for steps in (0, 1, 70):               # 70: one 64-step graph plus single steps
        g.step(steps - g.step_count)
        o.step(steps - o.step_count)
        err_e, err_q = _errs(g.moments(), o.moments(), scale_e, scale_q)
        assert err_e <= tol and err_q <= tol, (steps, err_e, err_q)
        assert np.abs(g.populations() - o.f).max() / scale_f <= tol
    # total energy: the deviation sum, to the storage's precision
    n = int(np.prod(shape))
    assert abs((g.energy() - n) - (o.f.sum() - n)) <= tol * np.abs(e - 1.0).sum()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
def test_d3q14_mode_matches_mode_matrix_96cubed(precision, tol):
    """A Fourier mode on a 96^3 lattice over 300 steps against the exact
    14x14 mode map (Eqs. 13-16, 54)."""
    n = 96
    tau_N, tau_R = 1.7, 25.0
    tau, tau_r = lt.relaxation(tau_N, tau_R)
    m = (2, 1, 3)
    k = np.array([2 * np.pi * mi / n for mi in m])
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    A = 1e-3
    g = plbm.LatticeND(plbm.D3Q14, (n, n, n), tau_N, tau_R, precision=precision)
    g.init(1 + A * np.cos(ph))
    steps = 300
    g.step(steps)
    e, qg = g.moments()
    F0 = lt.equilibrium(lt.D3Q14, A, np.zeros(3)).astype(complex)
    Fn = np.linalg.matrix_power(lt.mode_matrix(lt.D3Q14, k, tau, tau_r), steps) @ F0
    amp_e = Fn.sum()
    expect = 1 + np.real(amp_e * np.exp(1j * ph))
    assert np.abs(e - expect).max() <= tol * A
    kap = lt.kappa(tau_r)
    amp_q = kap * (lt.D3Q14.c.T.astype(float) @ Fn)
    for a in range(3):
        np.testing.assert_allclose(qg[a], np.real(amp_q[a] * np.exp(1j * ph)),
                                   atol=tol * A, rtol=0)


def test_nd_errors_and_speed():
    with pytest.raises(plbm.LBMError) as ei:
        plbm.LatticeND(plbm.D3Q14, (4, 4, 4), 0.9, 10.0, precision="fp16")
    assert ei.value.status == plbm.EUNSUPPORTED
    with pytest.raises(plbm.LBMError) as ei:
        plbm.LatticeND(plbm.D3Q14, (4, 4, 4), -1.0, 10.0)
    assert ei.value.status == plbm.EINVAL
    assert plbm.LatticeND.lattice_speed(plbm.D3Q14) == pytest.approx(math.sqrt(0.6))
    assert plbm.LatticeND.lattice_speed(plbm.D1Q2) == pytest.approx(1 / math.sqrt(3))
    g = plbm.LatticeND(plbm.D1Q2, (64,), 1.0, 5.0)
    with pytest.raises(plbm.LBMError):
        g.step(1)                          # not initialised
    g.init(np.ones(64))
    with pytest.raises(plbm.LBMError):
        g.init(np.full(64, np.nan))


def test_d3q14_bench_configuration_light_cone():
    """The D3Q14 bench workload at its full size (512^3, x-directed sine mode
    plus seeded noise, FP32): sampled nodes after 12 steps against the oracle
    on periodic (2n+1)^3 light-cone windows (a node after n steps depends only
    on nodes within n cells)."""
    n3, n = 512, 12
    w = inputs.THROUGHPUT_8192
    speed = plbm.LatticeND.lattice_speed(plbm.D3Q14)
    tau_N, tau_R = w.kn_N * w.length * speed, w.kn_R * w.length * speed
    x = np.arange(n3, dtype=np.float64)
    e = np.empty((n3, n3, n3))
    e[...] = 1.0 + 1e-3 * np.sin(2 * np.pi * x / 512.0)
    e += inputs.uniform_noise(e.shape, 1e-6)
    g = plbm.LatticeND(plbm.D3Q14, (n3, n3, n3), tau_N, tau_R)
    g.init(e)
    g.step(n)
    ge, gq = g.moments()
    g.close()
    rng = np.random.default_rng(2)
    pts = [(n3 - 1, n3 - 1, n3 - 1), (0, 0, 0)] + \
        [tuple(int(v) for v in rng.integers(0, n3, 3)) for _ in range(10)]
    res = []
    for (z, y, xx) in pts:
        idx = [np.arange(c - n, c + n + 1) % n3 for c in (z, y, xx)]
        win = np.ascontiguousarray(e[np.ix_(*idx)])
        o = lt.Run(lt.D3Q14, win.shape, tau_N, tau_R)
        o.init(win)
        o.step(n)
        oe, oq = o.moments()
        res.append((ge[z, y, xx] - oe[n, n, n], np.abs(gq[:, z, y, xx] - oq[:, n, n, n]).max(),
                    abs(oe[n, n, n] - 1.0), np.abs(oq[:, n, n, n]).max()))
    res = np.array(res)
    err_e = np.abs(res[:, 0]).max() / res[:, 2].max()
    err_q = res[:, 1].max() / res[:, 3].max()
    assert err_e <= TOL["fp32"] and err_q <= TOL["fp32"], (err_e, err_q)
