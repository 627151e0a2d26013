"""The shipped proposal-network weights and their metadata (CPU).

The weights file holds the architecture the metadata names, finite FP32
parameters of the right shapes, and survives a save / load round trip bit
for bit. The network computes only through the library's CUDA kernels: on
CPU tensors it refuses instead of falling back."""
import json
import os

import numpy as np
import pytest

from paper_2508_06672_gb300.proposal import ProposalNet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2508_06672_gb300", "weights", "proposal_2000km.npz")


def test_weights_match_their_metadata():
    with open(WEIGHTS[:-4] + ".json") as f:
        meta = json.load(f)
    net = ProposalNet.load(WEIGHTS, device="cpu")
    assert net.channels == meta["network"] == [20, 32, 64, 128, 64, 1]
    assert net.tc  # trained with the tensor-core convolutions; load keeps that arithmetic
    for (w, b), ci, co in zip(net.state_numpy(), net.channels[:-1], net.channels[1:]):
        assert w.shape == (co, ci, 3, 3) and b.shape == (co,)
        assert np.all(np.isfinite(w)) and np.all(np.isfinite(b))
        assert np.abs(w).max() > 0.0
    ev = meta["evaluation"]
    assert ev["scenes"] == 200 and ev["recall"] >= 0.99 and ev["recall"] > ev["recall_coarse_sum"]


def test_save_load_round_trip(tmp_path):
    net = ProposalNet.load(WEIGHTS, device="cpu")
    p = tmp_path / "copy.npz"
    net.save(str(p))
    again = ProposalNet.load(str(p), device="cpu")
    assert again.channels == net.channels
    for (w0, b0), (w1, b1) in zip(net.state_numpy(), again.state_numpy()):
        assert np.array_equal(w0, w1) and np.array_equal(b0, b1)


def test_forward_refuses_cpu_tensors():
    import torch
    net = ProposalNet([20, 4, 1], device="cpu")
    with pytest.raises(ValueError):
        net.forward(torch.zeros((1, 20, 8, 8), dtype=torch.float32))
