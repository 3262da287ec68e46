"""Warm-start network: GPU forward/backward kernels against the FP64 CPU
reference, training, and the warm start's effect on batched solves."""
import math

import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm
from oracle import mlp as omlp

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


def test_warm_start_reaches_same_state_in_fewer_steps():
    # training data: steady states of short channels from the batched solver
    train = warmstart.channels(192, seed=21, nx=warmstart.TRAIN_NX, w_range=(16, 48))
    prof, steps, r, _ = warmstart.steady_profiles(train)
    assert np.all(r < 1e-8)
    ws = warmstart.WarmStart(seed=0, max_batch=256)
    hist = ws.train(warmstart.features(train), prof, steps=800, batch=192, lr=2e-3)
    assert hist[-1] < hist[0] / 50
    # held-out channels of full length 4W
    test = warmstart.channels(12, seed=99, w_range=(16, 48))
    cold_steps, cold_r, _, cold = warmstart.solve(test)
    warm_steps, warm_r, _, warm = warmstart.solve(test, ws.predict(test))
    assert np.all(cold_r < 1e-8) and np.all(warm_r < 1e-8)
    assert warm_steps.sum() < 0.6 * cold_steps.sum(), (warm_steps, cold_steps)
    # both runs end at the same steady state (energy is conserved, so the
    # warm start keeps the cold start's mean energy)
    for k in range(len(test)):
        ce, cq, _ = cold.moments(k)
        we, wq, _ = warm.moments(k)
        assert np.abs(we - ce).max() <= 1e-3 * np.abs(ce - ce.mean()).max()
        assert np.abs(wq - cq).max() <= 1e-3 * np.abs(cq).max()
