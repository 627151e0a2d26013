"""Learned proposal: a small convolutional network over coarse maps.

The network maps K coarse per-snapshot maps of the footprint (channels) to
one map of logits over the same cells; sigmoid(logit) is the belief that the
emitter sits in that cell. Every layer runs in the library's own kernels
(dg_nn_*), forward and backward, and training is plain Adam on the weighted
binary cross-entropy against a target map built from the true emitter
position. torch is used only to hold device memory.

Architecture: conv3x3-relu blocks, then a conv3x3 to one logit channel
(``channels`` = [C_in, c1, ..., 1]).

Arithmetic: ``tc=True`` runs the convolutions forward and backward on the
tensor cores (dg_nn_conv3x3_*_tc: BF16 activations and weights, FP32
accumulation); the master weights and Adam's moments stay FP32. ``tc=False``
uses the FP32 CUDA-core kernels (the parity reference).
"""
from __future__ import annotations

import math

import numpy as np

from . import dg


class ProposalNet:
    def __init__(self, channels, seed=0, device="cuda", tc=False):
        import torch
        self.tc = bool(tc)
        if len(channels) < 2 or channels[-1] != 1:
            raise ValueError("channels must run from the input channels to 1")
        self.torch = torch
        self.channels = list(channels)
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        self.params = []
        for ci, co in zip(channels[:-1], channels[1:]):
            # He-normal for the relu blocks; the last layer starts small
            std = math.sqrt(2.0 / (9 * ci))
            w = rng.standard_normal((co, ci, 3, 3)) * std
            b = np.zeros(co)
            self.params.append([torch.tensor(w, dtype=torch.float32, device=self.device),
                                torch.tensor(b, dtype=torch.float32, device=self.device)])
        self.grads = [[torch.zeros_like(w), torch.zeros_like(b)] for w, b in self.params]
        self.m = [[torch.zeros_like(w), torch.zeros_like(b)] for w, b in self.params]
        self.v = [[torch.zeros_like(w), torch.zeros_like(b)] for w, b in self.params]
        self.t = 0
        self._acts = None

    # ---------------------------------------------------------------- state
    def state_numpy(self):
        return [(w.double().cpu().numpy(), b.double().cpu().numpy()) for w, b in self.params]

    def load_numpy(self, params):
        for (w, b), (wn, bn) in zip(self.params, params):
            w.copy_(self.torch.as_tensor(np.asarray(wn), dtype=self.torch.float32))
            b.copy_(self.torch.as_tensor(np.asarray(bn), dtype=self.torch.float32))

    def save(self, path):
        arrs = {}
        for k, (w, b) in enumerate(self.state_numpy()):
            arrs[f"w{k}"], arrs[f"b{k}"] = w.astype(np.float32), b.astype(np.float32)
        np.savez(path, channels=np.array(self.channels), tc=np.array(int(self.tc)), **arrs)

    @classmethod
    def load(cls, path, device="cuda", tc=None):
        """tc=None: the arithmetic the weights were trained with (stored)."""
        z = np.load(path)
        if tc is None:
            tc = bool(int(z["tc"])) if "tc" in z.files else False
        net = cls([int(c) for c in z["channels"]], device=device, tc=tc)
        net.load_numpy([(z[f"w{k}"], z[f"b{k}"]) for k in range(len(net.params))])
        return net

    # ------------------------------------------------------------- compute
    def forward(self, x, keep=False):
        """Logits (B, 1, H, W) for x (B, C_in, H, W), float32 CUDA. keep=True
        holds the activations for backward()."""
        torch = self.torch
        B, _, H, W = x.shape
        acts = [x]
        h = x
        L = len(self.params)
        for k, (w, b) in enumerate(self.params):
            z = torch.empty((B, w.shape[0], H, W), dtype=torch.float32, device=x.device)
            (dg.dg_nn_conv3x3_forward_tc if self.tc else dg.dg_nn_conv3x3_forward)(h, w, b, z)
            if k < L - 1:
                hk = torch.empty_like(z) if keep else z
                dg.dg_nn_relu_forward(z, hk)
                if keep:
                    acts += [z, hk]
                h = hk
            else:
                if keep:
                    acts.append(z)
                h = z
        self._acts = acts if keep else None
        return h

    def backward(self, dlogits):
        """Fill self.grads from the gradient of the loss wrt the logits of the
        last forward(keep=True)."""
        torch = self.torch
        acts = self._acts
        if acts is None:
            raise RuntimeError("backward() needs forward(..., keep=True) first")
        L = len(self.params)
        d = dlogits.contiguous()
        for k in range(L - 1, -1, -1):
            if k < L - 1:
                dz = torch.empty_like(d)
                dg.dg_nn_relu_backward(acts[2 * k + 1], d, dz)
                d = dz
            x = acts[2 * k]
            dx = torch.empty_like(x) if k > 0 else None
            (dg.dg_nn_conv3x3_backward_tc if self.tc else dg.dg_nn_conv3x3_backward)(
                x, self.params[k][0], d, dx, self.grads[k][0], self.grads[k][1])
            d = dx
        return self.grads

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        for (w, b), (gw, gb), (mw, mb), (vw, vb) in zip(self.params, self.grads, self.m, self.v):
            dg.dg_nn_adam(w, gw, mw, vw, lr, self.t, beta1, beta2, eps)
            dg.dg_nn_adam(b, gb, mb, vb, lr, self.t, beta1, beta2, eps)

    def loss_and_grad(self, logits, target, pos_weight):
        """Weighted BCE on logits (device scalar) and its gradient."""
        torch = self.torch
        grad = torch.empty_like(logits)
        loss = torch.empty(1, dtype=torch.float32, device=logits.device)
        dg.dg_nn_bce_logits(logits, target, pos_weight, grad, loss)
        return loss, grad

    def train_step(self, x, target, pos_weight, lr):
        logits = self.forward(x, keep=True)
        loss, grad = self.loss_and_grad(logits, target, pos_weight)
        self.backward(grad)
        self.adam_step(lr)
        self._acts = None
        return loss
