"""dg_set_grid and dg_search_regions: a context moved to another grid, or
searching several regions in turn, gives exactly what a context created on
that grid gives (same kernels, same captures)."""
import numpy as np
import pytest

import sim
from gpu_common import package, torch_cuda

pytestmark = pytest.mark.gpu


def _scene():
    return sim.make_scene(seed=31, fs_hz=5e6, n_samples=4096, k_steps=3, fmt="ci16", waveform="noise",
                          snr_db=-3.0, grid_n=41, grid_spacing_m=1000.0, bw_hz=4e6,
                          formation=sim.Formation(dt_s=5.0))


def _shifted(grid, di_m, dj_m, n=None):
    from paper_2508_06672_gb300.learned import degrees_per_metre
    dlat, dlon = degrees_per_metre(grid["lat0_deg"])
    g = dict(grid, lat0_deg=grid["lat0_deg"] + di_m * dlat, lon0_deg=grid["lon0_deg"] + dj_m * dlon)
    if n:
        g.update(nlat=n, nlon=n)
    return g


def _fresh(P, torch, s, grid, **opts):
    g = P.Geolocator(grid, s.ephem, s.fs_hz, s.fc_hz, **opts)
    g.load_captures(s.fmt, torch.from_numpy(s.y1).cuda(), torch.from_numpy(s.y2).cuda())
    return g


@pytest.mark.parametrize("opts", [dict(), dict(algo="cdft", contract="bf16x3")], ids=["direct", "cdft"])
def test_set_grid_equals_a_fresh_context(opts):
    torch = torch_cuda()
    P = package()
    s = _scene()
    g = _fresh(P, torch, s, s.grid, **opts)
    a0 = g.cost_surface().clone()
    other = _shifted(s.grid, 7000.0, -4000.0, n=57)  # larger: the ECEF buffer grows
    g.set_grid(other)
    b = g.cost_surface()
    f = _fresh(P, torch, s, other, **opts)
    assert torch.equal(b, f.cost_surface())
    g.set_grid(s.grid)
    assert torch.equal(g.cost_surface(), a0)
    g.close()
    f.close()


@pytest.mark.parametrize("opts", [dict(), dict(algo="cdft", contract="bf16x3")], ids=["direct", "cdft"])
def test_search_regions_matches_fresh_contexts(opts):
    torch = torch_cuda()
    P = package()
    s = _scene()
    regions = [_shifted(s.grid, di, dj, n=21) for di, dj in ((9000.0, 9000.0), (0.0, 0.0), (-8000.0, 5000.0))]
    g = _fresh(P, torch, s, s.grid, **opts)
    fix, best, costs = g.search_regions(regions, 100.0, 500.0)
    vals = []
    for r, reg in enumerate(regions):
        f = _fresh(P, torch, s, reg, **opts)
        c = f.cost_surface()
        assert torch.equal(costs[r], c)
        vals.append(float(c.max()))
        if r == best:
            ref = f.argmax_refine(c, 100.0, 500.0)
        f.close()
    assert best == int(np.argmax(vals))
    for k in ("i", "j", "lat_deg", "lon_deg", "cost", "refine_n", "ri", "rj", "refined_lat_deg",
              "refined_lon_deg", "refined_cost"):
        assert fix[k] == ref[k], k
    g.close()


def test_region_errors():
    torch = torch_cuda()
    P = package()
    s = _scene()
    g = _fresh(P, torch, s, s.grid)
    with pytest.raises(P.DGError, match="status 1"):
        g.search_regions([s.grid, dict(s.grid, nlat=11)])
    shard = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz, row0=3, nrows=10)
    with pytest.raises(P.DGError, match="status 6"):
        shard.set_grid(s.grid)
    shard.close()
    g.close()
