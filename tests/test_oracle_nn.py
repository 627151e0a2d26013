"""Pins of the proposal network's CPU oracle (oracle/nn.py) against library
routines and finite differences. CPU only."""
import numpy as np
import pytest
from scipy import signal

from oracle import nn


def _rand(rng, *shape):
    return rng.standard_normal(shape)


def test_conv3x3_is_scipy_correlate2d():
    """Forward: zero-padded 'same' 2-D cross-correlation summed over input
    channels, plus the bias (scipy.signal.correlate2d)."""
    rng = np.random.default_rng(1)
    x, w, b = _rand(rng, 2, 3, 7, 9), _rand(rng, 4, 3, 3, 3), _rand(rng, 4)
    y = nn.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(signal.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill") for c in range(3))
            assert np.allclose(y[n, o], want, rtol=1e-12, atol=1e-12)


def _fd(f, a, eps=1e-6):
    g = np.zeros_like(a)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = a[i]
        a[i] = old + eps
        fp = f()
        a[i] = old - eps
        fm = f()
        a[i] = old
        g[i] = (fp - fm) / (2 * eps)
    return g


def test_conv3x3_backward_finite_differences():
    rng = np.random.default_rng(2)
    x, w, b, g = _rand(rng, 2, 2, 5, 6), _rand(rng, 3, 2, 3, 3), _rand(rng, 3), _rand(rng, 2, 3, 5, 6)
    f = lambda: float(np.sum(g * nn.conv3x3(x, w, b)))
    dx, dw, db = nn.conv3x3_backward(x, w, g)
    assert np.allclose(dx, _fd(f, x), rtol=1e-6, atol=1e-7)
    assert np.allclose(dw, _fd(f, w), rtol=1e-6, atol=1e-7)
    assert np.allclose(db, _fd(f, b), rtol=1e-6, atol=1e-7)


def test_bce_logits_against_torch_and_finite_differences():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    z = _rand(rng, 2, 1, 4, 5) * 3
    t = (rng.uniform(size=z.shape) > 0.8).astype(float) * rng.uniform(size=z.shape)
    loss, grad = nn.bce_logits(z, t, pos_weight=7.0)
    want = torch.nn.functional.binary_cross_entropy_with_logits(
        torch.from_numpy(z), torch.from_numpy(t), pos_weight=torch.tensor(7.0, dtype=torch.float64))
    assert abs(loss - float(want)) < 1e-12
    assert np.allclose(grad, _fd(lambda: nn.bce_logits(z, t, 7.0)[0], z), rtol=1e-6, atol=1e-9)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    p0 = _rand(rng, 5, 3)
    grads = [_rand(rng, 5, 3) for _ in range(4)]
    tp = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for k, g in enumerate(grads, start=1):
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = nn.adam(p, g, m, v, k, 1e-2)
    assert np.allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_network_gradients_finite_differences():
    """Whole network (3 blocks): analytic gradients of the BCE loss equal
    finite differences of it, for every parameter."""
    rng = np.random.default_rng(5)
    chans = [1, 4, 3, 1]
    params = [(_rand(rng, chans[k + 1], chans[k], 3, 3) * 0.5, _rand(rng, chans[k + 1]) * 0.1) for k in range(3)]
    x = _rand(rng, 2, 1, 6, 5)
    t = np.zeros((2, 1, 6, 5))
    t[0, 0, 2, 3] = t[1, 0, 4, 1] = 1.0

    def loss():
        z, _ = nn.net_forward(params, x)
        return nn.bce_logits(z, t, 5.0)[0]

    z, acts = nn.net_forward(params, x)
    _, dz = nn.bce_logits(z, t, 5.0)
    grads = nn.net_backward(params, acts, dz)
    for (w, b), (dw, db) in zip(params, grads):
        assert np.allclose(dw, _fd(loss, w), rtol=1e-5, atol=1e-8)
        assert np.allclose(db, _fd(loss, b), rtol=1e-5, atol=1e-8)
