"""The N>1 path on CPU: two gloo ranks each evaluate their row block of a
grid with the oracle; the blocks concatenate to the unsharded surface and the
max-loc merge over ranks gives the unsharded argmax."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2508_06672_gb300.shard import merge_argmax, shard_rows


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    import sim

    return sim.make_scene(seed=41, fs_hz=5e6, n_samples=512, k_steps=2, fmt="ci16", waveform="noise",
                          snr_db=0.0, grid_n=(13, 9), grid_spacing_m=1500.0)


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import oracle
    from paper_2508_06672_gb300.shard import allreduce_argmax, shard_rows

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = _scene()
    r0, nr = shard_rows(s.grid["nlat"], world, rank)
    block = oracle.cost_surface(*oracle.scene_args(s), rows=(r0, r0 + nr))
    loc = int(np.argmax(block.ravel()))
    best = allreduce_argmax(block.ravel()[loc], r0 * s.grid["nlon"] + loc)
    q.put((rank, r0, block, best))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_rows_partition():
    for nlat in (1, 7, 1001, 2002):
        for world in (1, 2, 3, 8):
            if world > nlat:
                continue
            blocks = [shard_rows(nlat, world, r) for r in range(world)]
            assert blocks[0][0] == 0
            assert all(a[0] + a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            assert blocks[-1][0] + blocks[-1][1] == nlat
            assert max(b[1] for b in blocks) - min(b[1] for b in blocks) <= 1


def test_merge_argmax_rules():
    assert merge_argmax([(1.0, 5), (3.0, 9), (3.0, 2), (float("nan"), 0)]) == (3.0, 2)
    assert merge_argmax([(float("nan"), 1), (2.0, -1)])[1] == -1


def test_two_gloo_ranks_match_unsharded_oracle():
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = _scene()
    full = oracle.cost_surface(*oracle.scene_args(s))
    assert np.array_equal(np.concatenate([r[2] for r in res]), full)
    want = oracle.argmax(full)
    assert res[0][3] == res[1][3] == (float(full.ravel()[want]), want)
