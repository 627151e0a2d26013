"""The network's 3 x 3 convolution on the tensor cores (BF16 operands, FP32
accumulation) against the FP64 oracle (oracle/nn.py), forward and backward.

The bound is the arithmetic's own: each product rounds both operands to
BF16 (unit roundoff u = 2^-8), so it differs from the exact product by at
most (2u + u^2) |a| |b|; the products of BF16 values are exact in FP32, and
K of them summed in FP32 add at most K 2^-23 of the sum of the absolute
products. Every output is held to (2^-7 (1 + 2^-8) + K 2^-23) times the same
convolution over absolute values, computed by the oracle (the bias is added
in FP32: one more rounding of the result). The bias gradient rounds only dy:
u (1 + K 2^-15) of sum |dy|."""
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


def _bound(K):
    return 2.0 ** -7 * (1 + 2.0 ** -8) + K * 2.0 ** -23


# ragged shapes: channels that are not multiples of 16 and (channel, tap)
# counts that are not multiples of 32, widths beyond one 128-pixel tile,
# one-pixel images, more than 128 output channels (forward only)
SHAPES = [(2, 3, 5, 37, 45), (1, 20, 32, 9, 300), (3, 1, 1, 1, 1), (1, 64, 64, 6, 130), (2, 40, 8, 9, 3),
          (1, 7, 130, 5, 140)]


@pytest.mark.parametrize("shape", SHAPES)
def test_conv_tc_forward_within_the_bf16_bound(shape):
    P = package()
    torch = torch_cuda()
    B, Ci, Co, H, W = shape
    rng = np.random.default_rng(B * 1000 + Ci * 10 + Co)
    x = rng.standard_normal((B, Ci, H, W))
    w = rng.standard_normal((Co, Ci, 3, 3)) / np.sqrt(9 * Ci)
    b = rng.standard_normal(Co)
    xf, wf, bf = (np.asarray(a, np.float32).astype(np.float64) for a in (x, w, b))
    y = torch.empty((B, Co, H, W), dtype=torch.float32, device="cuda")
    P.dg_nn_conv3x3_forward_tc(_dev(xf), _dev(wf), _dev(bf), y)
    P.dg_nn_tc_check()
    ref = onn.conv3x3(xf, wf, bf)
    mag = onn.conv3x3(np.abs(xf), np.abs(wf), np.zeros(Co))
    lim = _bound(9 * Ci) * mag + 2.0 ** -23 * np.abs(ref) + 1e-30
    err = np.abs(_np(y) - ref)
    assert np.all(err <= lim), float(np.max(err / lim))
    # and the BF16 rounding is really there: not the FP32 result
    if Ci * Co > 1:
        assert np.max(err) > 0


@pytest.mark.parametrize("shape", [s for s in SHAPES if s[2] <= 128])
def test_conv_tc_backward_within_the_bf16_bound(shape):
    P = package()
    torch = torch_cuda()
    B, Ci, Co, H, W = shape
    rng = np.random.default_rng(7 + B * 1000 + Ci * 10 + Co)
    x = np.asarray(rng.standard_normal((B, Ci, H, W)), np.float32).astype(np.float64)
    w = np.asarray(rng.standard_normal((Co, Ci, 3, 3)) / np.sqrt(9 * Ci), np.float32).astype(np.float64)
    dy = np.asarray(rng.standard_normal((B, Co, H, W)), np.float32).astype(np.float64)
    dx = torch.empty((B, Ci, H, W), dtype=torch.float32, device="cuda")
    dw = torch.empty((Co, Ci, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.empty(Co, dtype=torch.float32, device="cuda")
    P.dg_nn_conv3x3_backward_tc(_dev(x), _dev(w), _dev(dy), dx, dw, db)
    P.dg_nn_tc_check()
    rdx, rdw, rdb = onn.conv3x3_backward(x, w, dy)
    mdx, mdw, _ = onn.conv3x3_backward(np.abs(x), np.abs(w), np.abs(dy))
    npix = B * H * W
    for got, ref, mag, K in ((dx, rdx, mdx, 9 * Co), (dw, rdw, mdw, npix)):
        lim = _bound(K) * mag + 1e-30
        err = np.abs(_np(got) - ref)
        assert np.all(err <= lim), float(np.max(err / lim))
    lim = 2.0 ** -8 * (1 + npix * 2.0 ** -15) * np.abs(dy).sum(axis=(0, 2, 3)) + 1e-30
    assert np.all(np.abs(_np(db) - rdb) <= lim)


def test_conv_tc_backward_is_deterministic_and_rejects_wide_outputs():
    P = package()
    torch = torch_cuda()
    rng = np.random.default_rng(3)
    B, Ci, Co, H, W = 2, 16, 24, 33, 70
    x, dy = (_dev(rng.standard_normal(s)) for s in ((B, Ci, H, W), (B, Co, H, W)))
    w = _dev(rng.standard_normal((Co, Ci, 3, 3)))
    outs = []
    for _ in range(2):
        dw = torch.empty((Co, Ci, 3, 3), dtype=torch.float32, device="cuda")
        db = torch.empty(Co, dtype=torch.float32, device="cuda")
        P.dg_nn_conv3x3_backward_tc(x, w, dy, None, dw, db)
        outs.append((dw.clone(), db.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    # more than 128 output channels: the scratch query gives the forward's
    # need only, and the backward's C entry point refuses with DG_EUNSUPPORTED
    import ctypes as C

    assert 0 < P.lib().dg_nn_conv3x3_tc_scratch(B, Ci, 130, H, W) < P.lib().dg_nn_conv3x3_tc_scratch(B, Ci, 128, H, W)
    wide = _dev(rng.standard_normal((130, Ci, 3, 3)))
    dyw = _dev(rng.standard_normal((B, 130, H, W)))
    dww, dbw, scr = torch.empty((130, Ci, 3, 3), device="cuda"), torch.empty(130, device="cuda"), torch.empty(16, device="cuda")
    st = P.lib().dg_nn_conv3x3_backward_tc(*(C.c_void_p(t.data_ptr()) for t in (x, wide, dyw)), None,
                                            *(C.c_void_p(t.data_ptr()) for t in (dww, dbw)), B, Ci, 130, H, W,
                                            C.c_void_p(scr.data_ptr()), None)
    assert st == P.DG_EUNSUPPORTED


def test_network_on_the_tensor_cores_tracks_the_oracle_and_trains():
    """The proposal network with every convolution on the tensor cores: its
    logits and gradients follow the FP64 oracle's chain rule, and Adam steps
    on a fixed batch lower the loss. Each layer is held to its BF16 rounding
    bound element by element above; here four stacked BF16 layers (measured:
    up to 7.6e-2 of a gradient tensor's largest value, 1e-2 on the logits)
    are held to 0.15, which a wrongly wired layer (an O(1) error) fails."""
    torch = torch_cuda()
    from paper_2508_06672_gb300.proposal import ProposalNet

    net = ProposalNet([6, 16, 24, 12, 1], seed=7, tc=True)
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

    def close(got, ref, tol):
        scale = max(np.max(np.abs(ref)), 1e-30)
        err = np.max(np.abs(got - ref)) / scale
        assert err <= tol, f"max error {err:.3e} of scale {scale:.3e} > {tol}"

    close(_np(logits), ref_logits, 2e-2)
    assert abs(float(loss.item()) - ref_loss) <= 1e-2 * abs(ref_loss)
    for (gw, gb), (rw, rb) in zip(grads, ref_grads):
        close(_np(gw), rw, 0.15)
        close(_np(gb), rb, 0.15)

    net = ProposalNet([3, 8, 8, 1], seed=9, tc=True)
    rng = np.random.default_rng(10)
    xb = rng.standard_normal((4, 3, 32, 32))
    tb = (xb[:, :1] + xb[:, 1:2] > 1.5).astype(np.float64)
    xd, td = _dev(xb), _dev(tb)
    first = float(net.train_step(xd, td, 2.0, 1e-2).item())
    for _ in range(60):
        last = float(net.train_step(xd, td, 2.0, 1e-2).item())
    torch.cuda.synchronize()
    assert last < 0.5 * first, (first, last)
