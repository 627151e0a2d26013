"""The proposal network's layers on the device (dg_nn_*) against the FP64
oracle (oracle/nn.py), layer by layer and for the whole network's gradients.

Tolerances: the kernels accumulate in FP32. A sum of n products carries a
rounding error of at most about n * 2^-24 relative to the sum of the absolute
products (about sqrt(n) * 2^-24 in practice). Every comparison is scaled by
the largest magnitude of the oracle's result; 2e-5 covers the worst sums
here (n <= 9 * 40 = 360 in the convolutions, n <= 2 * 37 * 45 = 3330 in the
weight and bias reductions: 3330 * 6e-8 = 2e-4 worst case, observed errors
sit near sqrt(n) * 6e-8 = 3.5e-6) with margin; the whole-network gradient
stacks four layers of such sums and is held to 1e-4."""
import numpy as np
import pytest

from gpu_common import package, torch_cuda
from oracle import nn as onn

pytestmark = pytest.mark.gpu


def _dev(a):
    torch = torch_cuda()
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def _np(t):
    return t.double().cpu().numpy()


def _close(got, ref, tol):
    scale = max(np.max(np.abs(ref)), 1e-30)
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, f"max error {err:.3e} of scale {scale:.3e} > {tol}"


# ragged shapes: channel counts that are not multiples of the kernels'
# 8-channel blocks, odd image sizes, one-pixel images
SHAPES = [(2, 3, 5, 37, 45), (1, 9, 17, 16, 16), (3, 1, 1, 1, 1), (1, 20, 32, 7, 130), (2, 40, 8, 9, 3)]


def _conv_case(B, Ci, Co, H, W, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, Ci, H, W))
    w = rng.standard_normal((Co, Ci, 3, 3)) / np.sqrt(9 * Ci)
    b = rng.standard_normal(Co)
    dy = rng.standard_normal((B, Co, H, W))
    return [np.asarray(a, np.float32).astype(np.float64) for a in (x, w, b, dy)]


@pytest.mark.parametrize("shape", SHAPES)
def test_conv3x3_forward(shape):
    torch = torch_cuda()
    P = package()
    B, Ci, Co, H, W = shape
    x, w, b, _ = _conv_case(*shape, seed=1)
    y = torch.empty((B, Co, H, W), dtype=torch.float32, device="cuda")
    P.dg_nn_conv3x3_forward(_dev(x), _dev(w), _dev(b), y)
    _close(_np(y), onn.conv3x3(x, w, b), 2e-5)


@pytest.mark.parametrize("shape", SHAPES)
def test_conv3x3_backward(shape):
    torch = torch_cuda()
    P = package()
    B, Ci, Co, H, W = shape
    x, w, b, dy = _conv_case(*shape, seed=2)
    dx = torch.full((B, Ci, H, W), 7.0, device="cuda")
    dw = torch.full((Co, Ci, 3, 3), 7.0, device="cuda")
    db = torch.full((Co,), 7.0, device="cuda")
    P.dg_nn_conv3x3_backward(_dev(x), _dev(w), _dev(dy), dx, dw, db)
    rdx, rdw, rdb = onn.conv3x3_backward(x, w, dy)
    _close(_np(dx), rdx, 2e-5)
    _close(_np(dw), rdw, 2e-5)
    _close(_np(db), rdb, 2e-5)
    # dx = NULL skips the data gradient and leaves the weight gradients equal
    dw2, db2 = torch.empty_like(dw), torch.empty_like(db)
    P.dg_nn_conv3x3_backward(_dev(x), _dev(w), _dev(dy), None, dw2, db2)
    assert torch.equal(dw2, dw) and torch.equal(db2, db)


def test_conv_is_deterministic():
    torch = torch_cuda()
    P = package()
    x, w, b, dy = _conv_case(2, 16, 24, 64, 64, seed=3)
    outs = []
    for _ in range(2):
        dx, dw, db = torch.empty((2, 16, 64, 64), device="cuda"), torch.empty((24, 16, 3, 3), device="cuda"), \
            torch.empty(24, device="cuda")
        P.dg_nn_conv3x3_backward(_dev(x), _dev(w), _dev(dy), dx, dw, db)
        outs.append((dx, dw, db))
    assert all(torch.equal(a, c) for a, c in zip(*outs))


def test_relu_forward_backward():
    torch = torch_cuda()
    P = package()
    rng = np.random.default_rng(4)
    z = np.asarray(rng.standard_normal(10007), np.float32).astype(np.float64)
    z[:5] = 0.0
    dh = rng.standard_normal(10007)
    zt, h, dz = _dev(z), torch.empty(10007, device="cuda"), torch.empty(10007, device="cuda")
    P.dg_nn_relu_forward(zt, h)
    P.dg_nn_relu_backward(zt, _dev(dh), dz)
    assert np.array_equal(_np(h), onn.relu(z))
    assert np.array_equal(_np(dz), onn.relu_backward(z, np.asarray(dh, np.float32).astype(np.float64)))


@pytest.mark.parametrize("n,pw", [(1, 1.0), (1000, 1.0), (262144 + 17, 50.0)])
def test_bce_logits(n, pw):
    torch = torch_cuda()
    P = package()
    rng = np.random.default_rng(5)
    z = np.asarray(rng.standard_normal(n) * 4.0, np.float32).astype(np.float64)
    z[:min(n, 3)] = [30.0, -30.0, 0.0][:min(n, 3)]
    t = (rng.uniform(size=n) < 0.1).astype(np.float64)
    t[: min(n, 2)] = [1.0, 0.0][: min(n, 2)]
    grad, loss = torch.empty(n, device="cuda"), torch.empty(1, device="cuda")
    P.dg_nn_bce_logits(_dev(z), _dev(t), pw, grad, loss)
    rl, rg = onn.bce_logits(z, t, pw)
    assert abs(float(loss.item()) - rl) <= 1e-5 * max(1.0, abs(rl))
    _close(_np(grad), rg, 1e-5)


def test_adam_matches_the_oracle_over_steps():
    torch = torch_cuda()
    P = package()
    rng = np.random.default_rng(6)
    p = np.asarray(rng.standard_normal(4099), np.float32).astype(np.float64)
    pd, md, vd = _dev(p), torch.zeros(4099, device="cuda"), torch.zeros(4099, device="cuda")
    m = np.zeros(4099)
    v = np.zeros(4099)
    for step in range(1, 6):
        g = np.asarray(rng.standard_normal(4099), np.float32).astype(np.float64)
        P.dg_nn_adam(pd, _dev(g), md, vd, 1e-2, step)
        p, m, v = onn.adam(p, g, m, v, step, 1e-2)
    _close(_np(pd), p, 1e-6)
    _close(_np(md), m, 1e-6)
    # beta2 reaches the kernel as the float nearest 0.999, so 1 - beta2 is
    # 0.00099998713: v sits 1.3e-5 (relative) below the FP64 oracle's
    _close(_np(vd), v, 3e-5)


def test_errors_are_reported():
    torch = torch_cuda()
    P = package()
    x = torch.zeros((1, 2, 4, 4), device="cuda")
    with pytest.raises(ValueError):
        P.dg_nn_conv3x3_forward(x, torch.zeros((3, 5, 3, 3), device="cuda"), torch.zeros(3, device="cuda"),
                                torch.zeros((1, 3, 4, 4), device="cuda"))
    L = P.lib()
    st = L.dg_nn_conv3x3_forward(None, None, None, None, 1, 1, 1, 1, 1, None)
    assert st == P.DG_EINVAL and "null" in P.dg_nn_last_error()
    st = L.dg_nn_adam(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 1e-3, 0.9, 0.999, 1e-8, 0, None)
    assert st == P.DG_EINVAL and "step" in P.dg_nn_last_error()


def test_network_gradients_match_the_oracle():
    """Whole network (4 conv blocks): logits, loss and every parameter
    gradient from the device's forward and backward kernels against the
    oracle's chain rule, on the same FP32-representable weights and input."""
    torch_cuda()
    from paper_2508_06672_gb300.proposal import ProposalNet

    net = ProposalNet([6, 16, 24, 12, 1], seed=7)
    params = net.state_numpy()
    rng = np.random.default_rng(8)
    x = np.asarray(rng.standard_normal((2, 6, 23, 29)), np.float32).astype(np.float64)
    t = (rng.uniform(size=(2, 1, 23, 29)) < 0.05).astype(np.float64)
    logits = net.forward(_dev(x), keep=True)
    loss, grad = net.loss_and_grad(logits, _dev(t), 20.0)
    grads = net.backward(grad)

    ref_logits, acts = onn.net_forward(params, x)
    ref_loss, ref_dz = onn.bce_logits(ref_logits, t, 20.0)
    ref_grads = onn.net_backward(params, acts, ref_dz)
    _close(_np(logits), ref_logits, 2e-5)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    for (gw, gb), (rw, rb) in zip(grads, ref_grads):
        _close(_np(gw), rw, 1e-4)
        _close(_np(gb), rb, 1e-4)


def test_training_reduces_the_loss():
    """A few Adam steps of the device network on a fixed batch lower the loss
    (the optimiser, the gradients and their signs work together)."""
    torch = torch_cuda()
    from paper_2508_06672_gb300.proposal import ProposalNet

    net = ProposalNet([3, 8, 8, 1], seed=9)
    rng = np.random.default_rng(10)
    x = rng.standard_normal((4, 3, 32, 32))
    t = (x[:, :1] + x[:, 1:2] > 1.5).astype(np.float64)
    xd, td = _dev(x), _dev(t)
    first = float(net.train_step(xd, td, 2.0, 1e-2).item())
    for _ in range(60):
        last = float(net.train_step(xd, td, 2.0, 1e-2).item())
    torch.cuda.synchronize()
    assert last < 0.5 * first, (first, last)
