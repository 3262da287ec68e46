"""Warm-start network: GPU forward/backward kernels against the FP64 CPU
reference, training, and the warm start's effect on batched solves."""
import math

import numpy as np
import pytest

import oracle
import paper_2010_01847_gb300 as plbm
from oracle import mlp as omlp
from oracle import update_matrix as um

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2010_01847_gb300 import warmstart  # noqa: E402


def bf16(a):
    """Round float values to bfloat16 (round to nearest even), as float64."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def _rounded_params(net, p):
    """Weights rounded to BF16 as the kernels use them; biases stay FP32."""
    out = p.astype(np.float64).copy()
    o = 0
    for k, n in zip(net.widths[:-1], net.widths[1:]):
        out[o:o + n * k] = bf16(p[o:o + n * k])
        o += n * k + n
    return out


@pytest.mark.parametrize("widths", [[3, 32, 24, 40], list(warmstart.WIDTHS)])
def test_forward_matches_oracle(widths):
    net = plbm.Mlp(widths, max_batch=256)
    net.init_params(seed=3)
    p = net.params()
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (200, widths[0])).astype(np.float32)
    y = net.forward(x).cpu().numpy()
    ref, _ = omlp.forward(_rounded_params(net, p), widths, bf16(x), hidden_round=bf16)
    scale = np.abs(ref).max()
    # FP32 accumulation vs FP64; a hidden value near a BF16 rounding boundary
    # may round the other way (one BF16 ulp, 2^-8 relative)
    assert np.abs(y - ref).max() <= 1e-2 * scale
    assert np.abs(y - ref).mean() <= 1e-3 * scale


def _grad_magnitudes(params, widths, x, t):
    """Per-element size of each gradient's products, for an element-wise
    bound: the backward pass of the FP64 reference run on absolute values,
    A_L = |dL/dy|, A_l = (A_{l+1} |W_{l+1}|) * |GELU'(z_l)|, and for layer l
    M_W = A_l^T |h_{l-1}|, M_b = sum over rows of A_l (same flat layout as
    the gradient)."""
    y, cache = omlp.forward(params, widths, x, hidden_round=bf16)
    layers = omlp.unpack(np.asarray(params, dtype=np.float64), widths)
    a = np.abs(2.0 * (y - np.asarray(t, dtype=np.float64)) / y.size)
    out = []
    for l in range(len(layers) - 1, -1, -1):
        h, z = cache[l]
        if l < len(layers) - 1:
            a = a * np.abs(omlp.gelu_grad(z))
        out.append((a.T @ np.abs(h), a.sum(0)))
        a = a @ np.abs(layers[l][0])
    flat = []
    for mw, mb in reversed(out):
        flat += [mw.ravel(), mb.ravel()]
    return np.concatenate(flat)


@pytest.mark.parametrize("widths", [[3, 32, 24, 40], list(warmstart.WIDTHS)])
def test_gradients_match_oracle(widths):
    net = plbm.Mlp(widths, max_batch=256)
    net.init_params(seed=5)
    p = net.params()
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (128, widths[0])).astype(np.float32)
    t = rng.normal(0, 1, (128, widths[-1])).astype(np.float32)
    loss, g = net.loss_grad(x, t)
    rp = _rounded_params(net, p)
    ref_loss, ref_g = omlp.loss_grad(rp, widths, bf16(x), t, hidden_round=bf16)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    # Element by element.  Each backward product takes BF16 operands (each
    # rounded by at most 2^-9 relative, so a product term by 2^-8), summed in
    # FP32; the error of a gradient element is then at most 2^-8 times the
    # sum of its terms' magnitudes, M, per layer it passes through, and the
    # incoming error dL/dy carries the forward pass's (one more layer).  With
    # L layers: |g - g_ref| <= (L + 1) 2^-8 M, plus an FP32 floor.  A wrong
    # index in any operand changes elements by O(M) and fails.
    m = _grad_magnitudes(rp, widths, bf16(x), t)
    L = len(widths) - 1
    bound = (L + 1) * 2.0 ** -8 * m + 1e-6 * np.abs(ref_g).max()
    excess = np.abs(g - ref_g) / bound
    assert excess.max() <= 1.0, (excess.max(), int(excess.argmax()))
    # and the bound is not vacuous: the typical element is far inside it
    assert np.median(np.abs(g - ref_g) / np.maximum(m, 1e-30)) < 2.0 ** -8


def test_training_reduces_loss():
    net = plbm.Mlp([3, 64, 64, 16], max_batch=512)
    net.init_params(seed=0)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (512, 3)).astype(np.float32)
    grid = np.linspace(0, 1, 16)
    t = np.sin(2.0 * x[:, :1] + 3.0 * grid[None, :] * x[:, 1:2]) * (1 + 0.5 * x[:, 2:3])
    t = t.astype(np.float32)
    first = net.train_step(x, t, 3e-3)
    for _ in range(400):
        last = net.train_step(x, t, 3e-3)
    assert last < first / 20, (first, last)
    assert np.isfinite(net.params()).all()


def test_device_training_loop_matches_step_by_step():
    """lbm_mlp_train (one captured Adam step replayed on the device) with the
    whole set as its minibatch and a constant learning rate takes the same
    steps as repeated lbm_mlp_train_step calls."""
    widths = [3, 32, 24, 40]
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (64, 3)).astype(np.float32)
    t = rng.normal(0, 1, (64, 40)).astype(np.float32)
    a = plbm.Mlp(widths, max_batch=64)
    a.init_params(seed=7)
    b = plbm.Mlp(widths, max_batch=64)
    b.set_params(a.params())
    hist = a.train(x, t, steps=25, batch=64, lr=2e-3, lr_final=2e-3)
    losses = [b.train_step(x, t, 2e-3) for _ in range(25)]
    np.testing.assert_allclose(hist, losses, rtol=1e-5)
    np.testing.assert_allclose(a.params(), b.params(), rtol=1e-4, atol=1e-6)
    # minibatches drawn on the device, cosine schedule: a smooth target is
    # learnt
    xs = rng.uniform(-1, 1, (512, 3)).astype(np.float32)
    grid = np.linspace(0, 1, 40)
    ts = (np.sin(2.0 * xs[:, :1] + 3.0 * grid[None, :] * xs[:, 1:2]) *
          (1 + 0.5 * xs[:, 2:3])).astype(np.float32)
    c = plbm.Mlp(widths, max_batch=64)
    c.init_params(seed=1)
    hist = c.train(xs, ts, steps=600, batch=64, lr=3e-3, lr_final=1e-4, seed=11)
    assert np.all(np.isfinite(hist)) and hist[-50:].mean() < hist[:10].mean() / 10


def test_analytic_profiles_follow_eq68():
    """lbm_analytic_profiles: Eq. 68 at Y = j/255 (written from the paper
    in the oracle's pins as a function of the Knudsen numbers), E = 0; ops
    add and subtract."""
    from tests.test_oracle_pins import eq68
    cases = [(16, 32, 0.01, 1.0), (8, 301, 0.01, 100.0), (24, 64, 0.1, 0.5), (8, 17, 1.0, 2.0)]
    inst = []
    for nx, ny, kn_N, kn_R in cases:
        d = ny - 1
        inst.append(dict(nx=nx, ny=ny, tau_N=plbm.tau_from_kn(kn_N, d),
                         tau_R=plbm.tau_from_kn(kn_R, d), bc_x=plbm.PERIODIC_GRADIENT,
                         bc_y=plbm.DIFFUSE_WALLS, delta_e=1e-3))
    prof = plbm.analytic_profiles(inst)
    p = prof.cpu().numpy()
    Y = np.arange(256) / 255
    for k, (_, _, kn_N, kn_R) in enumerate(cases):
        np.testing.assert_allclose(p[k, :256], eq68(Y, kn_N, kn_R), rtol=0, atol=2e-7)
        assert np.all(p[k, 256:] == 0.0)
    twice = plbm.analytic_profiles(inst, prof.clone(), op=1)
    assert torch.equal(twice, 2 * prof)
    zero = plbm.analytic_profiles(inst, prof.clone(), op=-1)
    assert torch.count_nonzero(zero).item() == 0
    with pytest.raises(plbm.LBMError):
        plbm.analytic_profiles([dict(inst[0], bc_y=plbm.PERIODIC)])


def _oracle_steady(inst):
    """The FP64 oracle's steady state of a channel, on its shortened copy
    (same gradient, warmstart.TRAIN_NX columns): the fixed point of the
    oracle's explicit one-step map T (f -> T [f; 1], oracle.update_matrix),
    solved directly with the total energy of the cold start, e = 1 at every
    node (the walled channel conserves it).  Returns (e, qx, qy)."""
    s = warmstart.shortened([inst])[0]
    nx, ny = s["nx"], s["ny"]
    p = oracle.params(s["tau_N"], s["tau_R"])
    T = um.step_matrix(nx, ny, p["tau"], p["tau_r"], s["bc_x"], s["bc_y"], s["delta_e"])
    n = 8 * nx * ny
    A = np.eye(n) - T[:n, :n]
    b = T[:n, n].copy()
    # one equation of the singular system (energy is conserved) replaced by
    # the total energy
    A[0, :] = 1.0
    b[0] = float(nx * ny)
    f = np.linalg.solve(A, b).reshape(ny, nx, 8)
    assert np.abs(T[:n, :n] @ f.ravel() + T[:n, n] - f.ravel()).max() < 1e-12
    o = oracle.Lattice(nx, ny, s["tau_N"], s["tau_R"], s["bc_x"], s["bc_y"], s["delta_e"])
    o.set_populations(f)
    return o.moments()


def _steady_errors(batch, k, inst, ref):
    """err_e, err_q of instance k's end state against the oracle's steady
    state (element by element on the full-length channel: q does not depend
    on x, e is the reference row profile plus the affine part with the
    steady slope -delta_e / nx)."""
    e, qx, qy = batch.moments(k)
    re, rqx, rqy = ref
    nx = inst["nx"]
    g = re.mean(axis=1) - re.mean()                     # row profile of e
    x = np.arange(nx) - 0.5 * (nx - 1)
    e_ref = re.mean() + g[:, None] - inst["delta_e"] / nx * x[None, :]
    q_ref = rqx.mean(axis=1)[:, None] * np.ones((1, nx))
    err_e = np.abs(e - e_ref).max() / np.abs(e_ref - e_ref.mean()).max()
    err_q = max(np.abs(qx - q_ref).max(), np.abs(qy).max()) / np.abs(q_ref).max()
    return err_e, err_q


def test_warm_start_reaches_the_steady_state_in_fewer_steps():
    # training data: steady states of short channels from the batched solver
    train = warmstart.channels(192, seed=21, nx=warmstart.TRAIN_NX, w_range=(16, 48))
    prof, steps, r, _ = warmstart.steady_profiles(train)
    assert np.all(r < 1e-8)
    ws = warmstart.WarmStart(seed=0, max_batch=256)
    hist = ws.train(train, prof, steps=800, batch=192, lr=2e-3)
    assert hist[-1] < hist[0] / 10
    # held-out channels of full length 4W, from three starts
    test = warmstart.channels(12, seed=99, w_range=(16, 32))
    cold_steps, cold_r, _, cold = warmstart.solve(test)
    ana_steps, ana_r, _, ana = warmstart.solve(test, warmstart.analytic_profiles(test))
    warm_steps, warm_r, _, warm = warmstart.solve(test, ws.predict(test))
    for r in (cold_r, ana_r, warm_r):
        assert np.all(r < 1e-8)
    assert warm_steps.sum() < 0.6 * cold_steps.sum(), (warm_steps, cold_steps)
    # the network learns the correction to Eq. 68: its start is closer to the
    # steady state than Eq. 68's alone, so it needs fewer steps
    assert warm_steps.sum() < ana_steps.sum(), (warm_steps, ana_steps)
    # every start ends at the true steady state (the FP64 oracle's), and the
    # learned start at least as close as the others: the solves stop at
    # r < 1e-8 over 100-step windows, which leaves the slowest mode at about
    # r / (its decay rate per step) of the state; 1e-3 bounds that for
    # channels of these widths (W <= 32), and FP32 storage adds ~1e-6
    errs = {"cold": [], "analytic": [], "learned": []}
    for k, inst in enumerate(test):
        ref = _oracle_steady(inst)
        for name, b in (("cold", cold), ("analytic", ana), ("learned", warm)):
            errs[name].append(_steady_errors(b, k, inst, ref))
    worst = {n: np.max(v) for n, v in errs.items()}
    assert all(w <= 1e-3 for w in worst.values()), worst
    assert worst["learned"] <= 2.0 * max(worst["cold"], worst["analytic"]) + 1e-6, worst
