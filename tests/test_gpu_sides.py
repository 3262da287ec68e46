"""GPU path with per-side boundary treatments (Section 2.5: isothermal
Eq. 55, heat flux Eqs. 56-57, diffuse Eq. 58 on any side, set through
lbm_set_side) against the FP64 oracle on the same seeded inputs, and the
paper's validation cases of Section 3 run on the GPU at the paper's grid
sizes against the continuum solutions in ``oracle.analytic``."""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic
import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs
from tests.helpers import TOL, check_gate, err_metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

S = plbm.SIDES
DIF, ISO, FLX = plbm.DIFFUSE, plbm.ISOTHERMAL, plbm.HEAT_FLUX
VG = math.sqrt(5.0 / 3.0)

# (name, nx, ny, bc_x, bc_y, delta_e, sides for left, right, bottom, top)
CASES = [
    ("film", 201, 3, S, plbm.PERIODIC, 0.0, [(ISO, 1.001), (ISO, 1.0), None, None]),
    ("square", 41, 41, S, S, 0.0, [(ISO, 1.0), (ISO, 1.0), (ISO, 1.0), (FLX, 1e-4)]),
    ("plate", 401, 3, S, plbm.PERIODIC, 0.0, [(FLX, 1e-4), (DIF, 0.0), None, None]),
    ("channel", 64, 20, plbm.PERIODIC_GRADIENT, S, 1e-3, [None, None, (ISO, 1.0005),
                                                          (FLX, -2e-4)]),
    ("walls_x_iso", 40, 12, S, plbm.DIFFUSE_WALLS, 0.0, [(ISO, 1.001), (ISO, 0.999), None,
                                                         None]),
    ("ragged", 37, 9, S, S, 0.0, [(ISO, 1.002), (ISO, 0.998), (FLX, 3e-4), (DIF, 0.0)]),
    ("y_diffuse", 48, 10, plbm.PERIODIC, S, 0.0, [None, None, (DIF, 0.0), (DIF, 0.0)]),
    ("tiny", 2, 2, S, S, 0.0, [(ISO, 1.001), (ISO, 1.0), (DIF, 0.0), (FLX, 1e-4)]),
]


def _oracle_sides(sides):
    # the oracle numbers the treatments as the C-ABI does; None = diffuse
    return [s if s is not None else (oracle.DIFFUSE, 0.0) for s in sides]


def _pair(case, precision, tau_N=0.9, tau_R=15.0, graph_chunk=None, seed=None, kernel="auto"):
    name, nx, ny, bcx, bcy, de, sides = case
    fields = inputs.random_state_fields(nx, ny, seed=seed or nx * 1000 + ny)
    g = plbm.Lattice(nx, ny, tau_N, tau_R, bcx, bcy, de, precision=precision,
                     graph_chunk=graph_chunk, kernel=kernel,
                     sides={i: s for i, s in enumerate(sides) if s is not None})
    g.init(*fields)
    o = oracle.Lattice(nx, ny, tau_N, tau_R, bcx, bcy, de, _oracle_sides(sides))
    o.init(*fields)
    return g, o


def _compare(g, o, precision):
    fo = np.moveaxis(o.f, 2, 0)
    dev = np.abs(fo - oracle.OMEGA[:, None, None] * fo.sum(0).mean()).max()
    err_f = np.abs(g.populations() - fo).max() / dev
    err_e, err_q = err_metrics(g.moments(), o.moments())
    return max(err_e, err_f), err_q


VEC = {"fp32": 4, "fp64": 2, "fp16": 8, "bf16": 8}


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16", "bf16"])
@pytest.mark.parametrize("kernel", ["scalar", "vector", "resident"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_sides_parity(case, kernel, precision):
    if kernel == "vector" and case[1] % VEC[precision]:
        pytest.skip(f"nx = {case[1]} is not a multiple of the vector width")
    if kernel == "resident" and precision != "fp32":
        pytest.skip("the cluster-resident kernel stores FP32")
    g, o = _pair(case, precision, kernel=kernel)
    assert g.kernel == kernel
    for steps in (1, 57):
        g.step(steps - g.step_count)
        o.step(steps - o.step_count)
        err_e, err_q = _compare(g, o, precision)

        def fp16_errors(steps=steps):
            f, fo = _pair(case, "fp16", kernel=kernel)
            f.step(steps)
            fo.step(steps)
            return _compare(f, fo, "fp16")

        check_gate(precision, err_e, err_q, fp16=fp16_errors)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_switched_pulse_matches_oracle_through_graphs(precision):
    """Section 3.4's time-switched side: heat flux for n_p steps, then
    diffuse.  With 8-step graphs, the switch must take effect at once."""
    case = CASES[2]
    g, o = _pair(case, precision, tau_N=0.3997, tau_R=4e5, graph_chunk=8)
    for n, switch in ((40, True), (150, False), (31, False)):
        g.step(n)
        o.step(n)
        err_e, err_q = _compare(g, o, precision)
        assert err_e <= TOL[precision] and err_q <= TOL[precision], (n, err_e, err_q)
        if switch:
            g.set_side(plbm.LEFT, DIF)
            o.set_side(0, oracle.DIFFUSE, 0.0)
            assert g.side(plbm.LEFT) == (DIF, 0.0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sides_residual_energy_and_fused_step(precision):
    case = CASES[1]
    g, o = _pair(case, precision)
    g.step(30)
    o.step(30)
    r0, en = g.residual()
    e_o = o.moments()[0]
    dev = np.abs(e_o - 1.0).sum()
    assert abs((en - e_o.size) - (e_o - 1.0).sum()) <= 1e-6 * dev
    # fused step + residual equals a plain step followed by the read-out
    r1, en1 = g.step_residual(10)
    o.step(10)
    e_o = o.moments()[0]
    assert abs((en1 - e_o.size) - (e_o - 1.0).sum()) <= 1e-6 * np.abs(e_o - 1.0).sum()
    assert math.isfinite(r1) and r1 > 0


def test_sides_checkpoint_round_trip():
    case = CASES[3]
    g, _ = _pair(case, "fp32")
    g.step(20)
    blob = g.get_state()
    g.step(25)
    ref = g.moments()
    g.set_state(blob)
    g.step(25)
    for a, b in zip(g.moments(), ref):
        np.testing.assert_array_equal(a, b)


def test_sides_vector_equals_scalar_bitwise():
    """The vector kernel's side treatment is the scalar kernel's, bit for bit
    (same arithmetic in the same order), through a switched side."""
    case = ("box", 96, 40, S, S, 0.0, [(ISO, 1.001), (ISO, 0.999), (FLX, 2e-4), (DIF, 0.0)])
    fields = inputs.random_state_fields(96, 40, seed=5)
    runs = []
    for kernel in ("scalar", "vector"):
        lat = plbm.Lattice(96, 40, 0.9, 15.0, S, S, 0.0, kernel=kernel, graph_chunk=8,
                           sides={i: s for i, s in enumerate(case[6])})
        lat.init(*fields)
        lat.step(20)
        lat.set_side(plbm.BOTTOM, DIF)
        r, en = lat.step_residual(21)
        runs.append((lat.populations(), lat.moments(), r, en))
    (fa, ma, ra, ea), (fb, mb, rb, eb) = runs
    assert np.array_equal(fa, fb)
    for x, y in zip(ma, mb):
        assert np.array_equal(x, y)
    # the residual step sums each node's terms over a warp in FP32, then in
    # FP64: the scalar kernel groups 32 single nodes, the vector kernel 32
    # vectors of 4, so the energies agree to the FP32 rounding of warp sums
    # of at most 128 terms, (128 - 1) 2^-24 sum |e - e_ref| (e_ref = 1)
    bound = 127 * 2.0 ** -24 * float(np.abs(ma[0] - 1.0).sum())
    assert abs(ea - eb) <= bound, (ea, eb, bound)
    assert rb == pytest.approx(ra, rel=1e-6)


def test_sides_kernel_choice_and_errors():
    # FP32 lattices of up to 16384 nodes run cluster-resident by default, FP64
    # ones one node per thread
    assert plbm.Lattice(64, 16, 0.9, 15.0, S, plbm.PERIODIC).kernel == "resident"
    assert plbm.Lattice(64, 16, 0.9, 15.0, S, plbm.PERIODIC, precision="fp64").kernel == "scalar"
    lat = plbm.Lattice(512, 64, 0.9, 15.0, S, plbm.PERIODIC)
    assert lat.kernel == "vector"                    # nx a multiple of the vector width
    with pytest.raises(plbm.LBMError) as ei:
        lat.set_kernel("staged")
    assert ei.value.status == plbm.EUNSUPPORTED
    lat.set_kernel("scalar")
    assert lat.kernel == "scalar"
    ragged = plbm.Lattice(517, 64, 0.9, 15.0, S, plbm.PERIODIC)
    assert ragged.kernel == "scalar"
    with pytest.raises(plbm.LBMError) as ei:
        ragged.set_kernel("vector")
    assert ei.value.status == plbm.EUNSUPPORTED
    with pytest.raises(plbm.LBMError) as ei:
        lat.set_side(plbm.BOTTOM, ISO, 1.0)          # y is periodic
    assert ei.value.status == plbm.EINVAL
    with pytest.raises(plbm.LBMError) as ei:
        lat.set_side(plbm.LEFT, 7, 1.0)
    assert ei.value.status == plbm.EINVAL
    with pytest.raises(plbm.LBMError) as ei:
        lat.set_side(plbm.LEFT, ISO, math.nan)
    assert ei.value.status == plbm.EINVAL
    lat.init(np.ones((64, 512)))
    lat.autotune(4)
    assert lat.kernel in ("scalar", "vector", "resident")
    # batches take periodic / gradient / walls only
    with pytest.raises(plbm.LBMError) as ei:
        plbm.Batch([dict(nx=64, ny=16, tau_N=0.9, tau_R=15.0, bc_x=S,
                         bc_y=plbm.DIFFUSE_WALLS)])
    assert ei.value.status == plbm.EUNSUPPORTED


def test_corner_without_isothermal_side_is_rejected():
    lat = plbm.Lattice(16, 8, 0.9, 15.0, S, plbm.DIFFUSE_WALLS)
    lat.init(np.ones((8, 16)))
    with pytest.raises(plbm.LBMError) as ei:
        lat.step(1)
    assert ei.value.status == plbm.EUNSUPPORTED
    lat.set_side(plbm.LEFT, ISO, 1.0)
    with pytest.raises(plbm.LBMError):
        lat.step(1)                                 # right corners still open
    lat.set_side(plbm.RIGHT, ISO, 1.0)
    lat.step(3)
    assert lat.step_count == 3


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_16bit_scale_covers_sides(precision):
    lat = plbm.Lattice(32, 3, 0.9, 15.0, S, plbm.PERIODIC, precision=precision,
                       sides=[(ISO, 1.5), (FLX, 0.02)])
    lat.init(np.ones((3, 32)))
    s = lat.storage_scale
    # the scale keeps |d_i| of the isothermal side (2/9 * 0.5) below 2^13
    assert (2 / 9) * 0.5 * s < 2 ** 13
    with pytest.raises(plbm.LBMError) as ei:
        lat.set_side(plbm.LEFT, ISO, 1.0 + 1e6)
    assert ei.value.status == plbm.EINVAL
    lat.step(10)
    e, _, _ = lat.moments()
    assert np.isfinite(e).all() and e[:, 0] == pytest.approx(1.5, rel=1e-3)


# --- the paper's cases at the paper's grids, against Section 3's solutions --------
def _run(nx, ny, tau_N, tau_R, bcx, bcy, sides, e0, steps, precision="fp32", switch=None):
    lat = plbm.Lattice(nx, ny, tau_N, tau_R, bcx, bcy, precision=precision,
                       sides={i: sd for i, sd in enumerate(sides) if sd is not None})
    lat.init(np.full((ny, nx), e0))
    if switch:
        n_p, side, kind = switch
        lat.step(n_p)
        lat.set_side(side, kind, 0.0)
    lat.step(steps - lat.step_count)
    return lat


def _l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_paper_film_201x3_eqs_61_64(precision):
    """Section 3.1.1 on the paper's 201 x 3 grid at t* = 1e6 (Fig. 4)."""
    N, d = 201, 200
    tau_N, tau_R = plbm.tau_from_kn(1.29e3, d), plbm.tau_from_kn(1.29e-3, d)
    steps = int(round(1e6 * tau_R))
    lat = _run(N, 3, tau_N, tau_R, S, plbm.PERIODIC,
               [(ISO, 1.001), (ISO, 1.0), None, None], 1.0, steps, precision)
    e, qx, _ = lat.moments()
    th_a, Q_a = analytic.fourier_transient_1d(np.arange(N) / d, steps / tau_R, 1.29e-3)
    theta = (e.mean(0) - 1.0) / 1e-3
    Q = qx.mean(0) * d / ((5 / 9) * tau_R * 1e-3)
    # the FP64 oracle gives 1.49e-3 and 1.29e-2 on this grid
    assert _l1(theta, th_a) < 2e-3 and _l1(Q, Q_a) < 0.015


def test_paper_square_201x201_eqs_65_67():
    """Section 3.1.2 on the paper's 201 x 201 grid, run to steady state."""
    N, L = 201, 200
    tau_N, tau_R = plbm.tau_from_kn(2e3, L), plbm.tau_from_kn(2e-3, L)
    k = 5 / 9 * tau_R
    q0 = 1e-4
    lat = _run(N, N, tau_N, tau_R, S, S, [(ISO, 1.0), (ISO, 1.0), (ISO, 1.0), (FLX, q0)],
               1.0, int(4 * L * L / k))
    e, qx, qy = lat.moments()
    Y, X = np.mgrid[0:N, 0:N] / L
    th_a, qx_a, qy_a = analytic.square_steady(X, Y)
    th = (e - 1.0) * k / (q0 * L)
    for frac in (0.25, 0.5, 0.75):           # the cross-sections of Fig. 5
        r = int(round(frac * L))
        # 41 x 41 gives up to 0.15, 81 x 81 up to 0.065 (first order)
        assert _l1(th[r], th_a[r]) < 0.03
        assert _l1(qx[r] / q0, qx_a[r]) < 0.035
        assert _l1(qy[r] / q0, qy_a[r]) < 0.03


@pytest.mark.parametrize("kn_R,tol_t,tol_q", [(0.01, 2e-3, 0.01), (1.0, 0.02, 0.15),
                                              (100.0, 2e-3, 0.2)])
def test_paper_cross_plane_301x3_eqs_70_71(kn_R, tol_t, tol_q):
    """Section 3.3 on the paper's 301 x 3 grid (Kn_N = 0.01)."""
    N, d = 301, 300
    lat = _run(N, 3, plbm.tau_from_kn(0.01, d), plbm.tau_from_kn(kn_R, d), S, plbm.PERIODIC,
               [(ISO, 1.001), (ISO, 1.0), None, None], 1.0, 100000)
    e, qx, _ = lat.moments()
    X = np.arange(N) / d
    th_a, Q_a = analytic.cross_plane(X, kn_R)
    theta = (e.mean(0) - 1.0) / 1e-3
    core = (X >= 0.1) & (X <= 0.9)
    assert np.abs(theta - th_a)[core].max() < tol_t
    assert (qx.mean(0)[1:-1] / (VG * 1e-3)).mean() == pytest.approx(Q_a, rel=tol_q)


@pytest.mark.parametrize("kn_R,tol_t,tol_q", [(1.29e3, 0.03, 0.03), (1.29, 0.025, 0.03),
                                              (1.29e-3, 3e-3, 0.05)])
def test_paper_heat_pulse_401x3_appendix_b(kn_R, tol_t, tol_q):
    """Section 3.4 on the paper's 401 x 3 grid: the pulse of 100 tau_N into
    the left side, then both sides adiabatic."""
    N, d = 401, 400
    tau_N, tau_R = plbm.tau_from_kn(1.29e-3, d), plbm.tau_from_kn(kn_R, d)
    n_p = int(round(100 * tau_N))
    q0 = 1e-4
    X = np.arange(N) / d
    for t_star in (300.0, 1200.0):
        steps = int(round(t_star * tau_N))
        lat = _run(N, 3, tau_N, tau_R, S, plbm.PERIODIC,
                   [(FLX, q0), (DIF, 0.0), None, None], 1.0, steps,
                   switch=(n_p, plbm.LEFT, DIF))
        e, qx, _ = lat.moments()
        th_a, Q_a = analytic.heat_pulse(X, steps / tau_N, 1.29e-3, kn_R, t_pulse=n_p / tau_N,
                                        gamma_t=9.0)
        assert _l1((e.mean(0) - 1.0) * VG / q0, th_a) < tol_t
        assert _l1(qx.mean(0) / q0, Q_a) < tol_q


@pytest.mark.parametrize("precision,tol,flat", [("fp64", 1e-4, 1e-3), ("fp32", 2e-3, 1e-2)])
def test_paper_heat_pulse_terminal_rise_401x3(precision, tol, flat):
    """Section 3.4: the diffusive plate settles at n_p v_g / d, i.e.
    100 Kn_N = 0.129 (Fig. 13 inset).  With FP32 storage the last slow
    mode stops decaying once its per-step change (1.4e-5 of its amplitude
    here) falls below the rounding of the populations: it stalls near 0.5 %
    of the rise (measured 0.6 %), hence the looser flatness bound."""
    N, d = 401, 400
    tau_N, tau_R = plbm.tau_from_kn(1.29e-3, d), plbm.tau_from_kn(1.29e-3, d)
    n_p = int(round(100 * tau_N))
    steps = n_p + int(3.5 * d * d / (5 / 9 * tau_R))
    lat = _run(N, 3, tau_N, tau_R, S, plbm.PERIODIC,
               [(FLX, 1e-4), (DIF, 0.0), None, None], 1.0, steps, precision,
               switch=(n_p, plbm.LEFT, DIF))
    theta = (lat.moments()[0] - 1.0) * VG / 1e-4
    assert np.ptp(theta) < flat * theta.mean()
    assert theta.mean() == pytest.approx(n_p * VG / d, rel=tol)
    assert theta.mean() == pytest.approx(0.129, rel=2e-3)
