"""Plain FP64 reference of the proposal network's layers (NumPy).

TEST INFRASTRUCTURE: only ``tests/`` may import this module. It is the CPU
oracle that the device's forward and backward kernels of the learned
proposal are checked against; it shares no code with them.

Layers (NCHW tensors, float64):

* ``conv3x3``: 3 x 3 cross-correlation with zero padding 1, stride 1, bias:
  y[n,o,i,j] = b[o] + sum_c sum_{u,v in -1..1} w[o,c,u+1,v+1] x[n,c,i+u,j+v];
* ``relu``;
* ``bce_logits``: binary cross-entropy of sigmoid(z) against targets t in
  [0, 1], with weight p for the positive term, averaged over all elements:
  L = mean(-p t log s(z) - (1 - t) log(1 - s(z)));
* ``adam``: one Adam step (Kingma & Ba, 2015) with bias correction.

Each backward function follows from the forward definition by the chain
rule; the pins check them against finite differences and library routines.
"""
from __future__ import annotations

import numpy as np


def _pad(x):
    return np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))


def conv3x3(x, w, b):
    """Forward: x (B, Ci, H, W), w (Co, Ci, 3, 3), b (Co,) -> (B, Co, H, W)."""
    B, Ci, H, W = x.shape
    xp = _pad(x)
    y = np.zeros((B, w.shape[0], H, W))
    for u in range(3):
        for v in range(3):
            # tap (u - 1, v - 1): x[n, c, i + u - 1, j + v - 1]
            y += np.einsum("oc,nchw->nohw", w[:, :, u, v], xp[:, :, u:u + H, v:v + W])
    return y + b[None, :, None, None]


def conv3x3_backward(x, w, dy):
    """Gradients of sum(dy * conv3x3(x, w, b)) with respect to x, w and b."""
    B, Ci, H, W = x.shape
    xp = _pad(x)
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for u in range(3):
        for v in range(3):
            dxp[:, :, u:u + H, v:v + W] += np.einsum("oc,nohw->nchw", w[:, :, u, v], dy)
            dw[:, :, u, v] = np.einsum("nohw,nchw->oc", dy, xp[:, :, u:u + H, v:v + W])
    return dxp[:, :, 1:1 + H, 1:1 + W], dw, dy.sum(axis=(0, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, dy):
    """Gradient of relu at x (the subgradient 0 is taken at x = 0)."""
    return dy * (x > 0.0)


def bce_logits(z, t, pos_weight=1.0):
    """Mean weighted binary cross-entropy of sigmoid(z) against t, and its
    gradient with respect to z."""
    z = np.asarray(z, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    log_s = -np.logaddexp(0.0, -z)        # log sigmoid(z)
    log_1ms = -np.logaddexp(0.0, z)       # log (1 - sigmoid(z))
    loss = np.mean(-pos_weight * t * log_s - (1.0 - t) * log_1ms)
    # dL/dz = (p t (s - 1) + (1 - t) s) / n, with s - 1 = -(1 - s) taken as
    # exp(log(1 - s)) so that it keeps its digits where s rounds to 1
    s, one_minus_s = np.exp(log_s), np.exp(log_1ms)
    grad = (-pos_weight * t * one_minus_s + (1.0 - t) * s) / z.size
    return loss, grad


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1): returns the new p, m, v."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def net_forward(params, x):
    """The proposal network: conv-relu blocks, then a final conv to one map
    of logits. params = [(w, b), ...]. Returns the logits and the tensors
    [x, z1, h1, z2, h2, ..., z_L] (z: conv outputs, h = relu(z)) that
    net_backward needs."""
    acts = [x]
    h = x
    L = len(params)
    for k, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        acts.append(z)
        if k < L - 1:
            h = relu(z)
            acts.append(h)
        else:
            h = z
    return h, acts


def net_backward(params, acts, dz_out):
    """Gradients [(dw, db), ...] of the network, given the gradient dz_out
    of the loss with respect to the logits. Layer k reads acts[2k] and
    produced acts[2k + 1]."""
    L = len(params)
    grads = [None] * L
    d = dz_out
    for k in range(L - 1, -1, -1):
        if k < L - 1:
            d = relu_backward(acts[2 * k + 1], d)
        dx, dw, db = conv3x3_backward(acts[2 * k], params[k][0], d)
        grads[k] = (dw, db)
        d = dx
    return grads
