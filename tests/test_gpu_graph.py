"""Whole steps replayed as CUDA graphs (dg_graph_*) and many uneven
captures as one graph (dg_batch_*): the fixes equal those of the
synchronising calls (dg_cost_surface + dg_argmax_refine) field for field,
on the same inputs, for both evaluations of Eq. 11."""
import numpy as np
import pytest

import sim
from gpu_common import package, torch_cuda

pytestmark = pytest.mark.gpu

REFINE = (10.0, 200.0)


def _geo(scene, stream, **opts):
    torch = torch_cuda()
    P = package()
    g = P.Geolocator(scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz, stream=stream, **opts)
    g.load_captures(scene.fmt, torch.from_numpy(scene.y1).cuda(), torch.from_numpy(scene.y2).cuda())
    return g


def _reference_fix(g, refine=REFINE):
    with g.torch.cuda.stream(g.stream):
        c = g.cost_surface()
        return c, g.argmax_refine(c, *refine)


def _scene(seed, **kw):
    args = dict(seed=seed, fs_hz=12.5e6, n_samples=20000, k_steps=4, fmt="ci16", waveform="chirp", snr_db=-5.0,
                grid_n=(121, 131), grid_spacing_m=200.0)
    args.update(kw)
    return sim.make_scene(**args)


ALGOS = [dict(), dict(algo="cdft", contract="fp16x3")]


@pytest.mark.parametrize("opts", ALGOS, ids=["direct", "cdft"])
def test_graph_fix_equals_synchronous_step(opts):
    torch = torch_cuda()
    s = _scene(31)
    stream = torch.cuda.Stream()
    g = _geo(s, stream, **opts)
    ref_cost, ref = _reference_fix(g)
    cost = torch.empty_like(ref_cost)
    g.graph_capture(cost, *REFINE)
    for _ in range(3):
        g.graph_launch()
    fix = g.graph_fix()
    assert fix == ref
    stream.synchronize()
    assert torch.equal(cost, ref_cost)
    g.close()


@pytest.mark.parametrize("opts", ALGOS, ids=["direct", "cdft"])
def test_graph_replays_reloaded_captures(opts):
    """New captures of the same formats and lengths feed the captured graph;
    its fix equals the synchronising step on the new data."""
    torch = torch_cuda()
    a, b = _scene(32), _scene(33)
    stream = torch.cuda.Stream()
    g = _geo(a, stream, **opts)
    cost = torch.empty((g.nrows, g.nlon), dtype=g.dtype, device=g.device)
    g.graph_capture(cost, *REFINE)
    g.load_captures(b.fmt, torch.from_numpy(b.y1).cuda(), torch.from_numpy(b.y2).cuda())
    g.graph_launch()
    fix_b = g.graph_fix()
    _, ref_b = _reference_fix(g)
    assert fix_b == ref_b
    g.close()


def test_graph_state_errors():
    torch = torch_cuda()
    P = package()
    s = _scene(34, k_steps=2)
    stream = torch.cuda.Stream()
    g = _geo(s, stream)
    with pytest.raises(P.DGError):
        g.graph_launch()  # nothing captured yet
    cost = torch.empty((g.nrows, g.nlon), dtype=g.dtype, device=g.device)
    g.graph_capture(cost)
    g.graph_launch()
    assert g.graph_fix()["refine_n"] == 0
    # a different length changes the captured buffers' shape: refused
    g.load_capture(0, s.fmt, torch.from_numpy(s.y1[0][:15000].copy()).cuda(),
                   torch.from_numpy(s.y2[0][:15000].copy()).cuda())
    with pytest.raises(P.DGError) as e:
        g.graph_launch()
    assert e.value.status == P.DG_ESTATE
    g.close()
    # a context on the default stream cannot be captured
    d = _geo(s, None)
    with pytest.raises(P.DGError) as e:
        d.graph_capture(torch.empty((d.nrows, d.nlon), dtype=d.dtype, device=d.device))
    assert e.value.status == P.DG_EUNSUPPORTED
    d.close()


def test_batch_of_uneven_captures():
    """Six independent problems with different grids, snapshot counts,
    lengths, formats and algorithms in one graph: every fix equals its own
    synchronising step."""
    torch = torch_cuda()
    P = package()
    rng = np.random.default_rng(5)
    gs, costs, refs = [], [], []
    for i in range(6):
        fmt = ["ci16", "ci8", "c64"][i % 3]
        s = _scene(40 + i, fmt=fmt, k_steps=int(rng.integers(1, 5)), n_samples=int(rng.choice([4096, 9000, 16384])),
                   grid_n=(int(rng.integers(31, 90)) | 1, int(rng.integers(31, 90)) | 1),
                   grid_spacing_m=float(rng.uniform(100, 400)), waveform=["chirp", "noise"][i % 2])
        g = _geo(s, torch.cuda.Stream(), **ALGOS[i % 2])
        _, ref = _reference_fix(g)
        gs.append(g)
        refs.append(ref)
        costs.append(torch.empty((g.nrows, g.nlon), dtype=g.dtype, device=g.device))
    b = P.Batch(gs, costs, *REFINE)
    assert b.launch_count() > 6
    for _ in range(2):
        b.launch()
    assert b.fixes() == refs
    b.close()
    for g in gs:
        g.close()


def test_batch_shares_tensor_core_contraction_rounds():
    """Seven uneven chunked-DFT problems on the tensor cores (one format):
    their main-surface contractions run as shared persistent launches, one
    per round of snapshot batches (a context with a small scratch target
    splits its snapshots over several rounds). Every fix and cost surface
    equals its own synchronising step bit for bit, and one capture's
    surface matches the CPU oracle."""
    torch = torch_cuda()
    P = package()
    import oracle
    from gpu_common import lag_boundary_mask, rel_err

    rng = np.random.default_rng(6)
    gs, costs, refs, ref_costs, scenes = [], [], [], [], []
    for i in range(7):
        k = int(rng.integers(1, 6))
        s = _scene(60 + i, fmt="ci16", k_steps=4 if i == 6 else k,
                   n_samples=int(rng.choice([4096, 9000, 16384, 20000])),
                   grid_n=(int(rng.integers(31, 90)) | 1, int(rng.integers(31, 90)) | 1),
                   grid_spacing_m=float(rng.uniform(100, 400)), waveform=["chirp", "noise"][i % 2])
        # the last context keeps one snapshot per batch of its plan: several rounds
        opts = dict(algo="cdft", contract="fp16x3", scratch_mib=1 if i == 6 else 0)
        g = _geo(s, torch.cuda.Stream(), **opts)
        c, ref = _reference_fix(g)
        g.stream.synchronize()
        ref_costs.append(c.clone())
        gs.append(g)
        refs.append(ref)
        scenes.append(s)
        costs.append(torch.empty((g.nrows, g.nlon), dtype=g.dtype, device=g.device))
    b = P.Batch(gs, costs, *REFINE)
    assert b.rounds() >= 2
    for _ in range(2):
        b.launch()
    assert b.fixes() == refs
    torch.cuda.synchronize()
    for c, rc in zip(costs, ref_costs):
        assert torch.equal(c, rc)
    s = scenes[0]
    ref = oracle.cost_surface(*oracle.scene_args(s))
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(costs[0].double().cpu().numpy().ravel()[ok], ref.ravel()[ok], 0.01) < 1e-4
    b.close()
    for g in gs:
        g.close()


@pytest.mark.parametrize("contract", ["fp32", "fp16x3"])
def test_autotune_picks_an_admissible_shape(contract):
    """The tuner times the admissible (chunk, tile) shapes, keeps the fastest
    in the context, and caches it; the tuned context's surface equals one
    created with that shape explicitly, bit for bit."""
    torch = torch_cuda()
    s = _scene(50, k_steps=3, n_samples=30000)
    g = _geo(s, torch.cuda.Stream(), algo="cdft", contract=contract)
    t = g.autotune(reps=2)
    assert 256 <= t["chunk"] <= 16384 and t["chunk"] & (t["chunk"] - 1) == 0
    assert t["tiles"] in (1, 2) and (contract != "fp32" or t["tiles"] == 1)
    assert t["cached"] == 0 and t["tried"] >= 3 and t["ms"] > 0
    with torch.cuda.stream(g.stream):
        tuned = g.cost_surface().clone()
    tiles = {1: "rows", 2: "lags"}[t["tiles"]]
    h = _geo(s, torch.cuda.Stream(), algo="cdft", contract=contract, chunk=t["chunk"], tiles=tiles)
    with torch.cuda.stream(h.stream):
        explicit = h.cost_surface().clone()
    torch.cuda.synchronize()
    assert torch.equal(tuned, explicit)
    # a second context of the same shape takes the cached choice
    u = _geo(s, torch.cuda.Stream(), algo="cdft", contract=contract)
    t2 = u.autotune()
    assert t2["cached"] == 1 and (t2["chunk"], t2["tiles"]) == (t["chunk"], t["tiles"])
    for x in (g, h, u):
        x.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,delay", [("fp32", "integer"), ("fp32", "lagrange4"), ("fp64", "integer")])
def test_direct_rows_per_thread_are_tuned_and_bit_identical(prec, delay):
    """The direct kernel's grid rows per thread change only the tile shape:
    every admissible value gives the same surface bit for bit (each
    candidate's arithmetic is its own), the tuner picks one of them and
    caches it, and a value outside the admissible set is rejected."""
    torch = torch_cuda()
    P = package()
    s = _scene(51, k_steps=2, n_samples=6000)
    rows = {"fp32": (4, 8, 16), "fp64": (2, 4)}[prec]
    surfs = []
    for r in rows:
        g = _geo(s, torch.cuda.Stream(), prec=prec, delay=delay, rows=r)
        with torch.cuda.stream(g.stream):
            surfs.append(g.cost_surface().clone())
        torch.cuda.synchronize()
        g.close()
    for x in surfs[1:]:
        assert torch.equal(x, surfs[0])
    g = _geo(s, torch.cuda.Stream(), prec=prec, delay=delay)
    t = g.autotune(reps=2)
    tried = rows if (prec == "fp64" or delay == "integer") else (4, 8)
    assert t["rows"] in tried and t["tried"] == len(tried) and t["cached"] == 0 and t["ms"] > 0
    assert t["chunk"] == 0 and t["tiles"] == 0
    with torch.cuda.stream(g.stream):
        tuned = g.cost_surface().clone()
    torch.cuda.synchronize()
    assert torch.equal(tuned, surfs[0])
    u = _geo(s, torch.cuda.Stream(), prec=prec, delay=delay)
    t2 = u.autotune()
    assert t2["cached"] == 1 and t2["rows"] == t["rows"]
    for x in (g, u):
        x.close()
    bad = 16 if prec == "fp64" else 2
    with pytest.raises(P.DGError):
        _geo(s, torch.cuda.Stream(), prec=prec, delay=delay, rows=bad)
