"""Host-side geometry of the learned search and its training examples (CPU).

The coarse maps cover the footprint with cells x cells cells whose corners
are the nodes of a (cells + 1)^2 grid and whose centres form a cells^2 grid;
node_of inverts the grid's node formula (WGS-84 radii at the centre
latitude); cell_of picks the cell holding a point; the training target is a
Gaussian bump of peak 1 on the emitter's cell and the crops keep it inside
the window."""
import math

import numpy as np

import sim
from paper_2508_06672_gb300 import learned as L
from paper_2508_06672_gb300 import training

A, F = 6378137.0, 1.0 / 298.257223563


def _node_deg(grid, i, j):
    e2 = F * (2.0 - F)
    lat0 = math.radians(grid["lat0_deg"])
    w = math.sqrt(1.0 - e2 * math.sin(lat0) ** 2)
    m, n = A * (1.0 - e2) / w ** 3, A / w
    lat = lat0 + (i - 0.5 * (grid["nlat"] - 1)) * grid["dlat_m"] / m
    lon = math.radians(grid["lon0_deg"]) + (j - 0.5 * (grid["nlon"] - 1)) * grid["dlon_m"] / (n * math.cos(lat0))
    return math.degrees(lat), math.degrees(lon)


def test_footprint_grids_cover_the_footprint():
    g = sim.learned(5).grid
    nodes, centres = L.footprint_grids(g, 512)
    assert (nodes["nlat"], nodes["nlon"], centres["nlat"], centres["nlon"]) == (513, 513, 512, 512)
    # the cell grid's corner nodes are the full grid's corners
    for (a, b), (fa, fb) in (((0, 0), (0, 0)), ((512, 512), (g["nlat"] - 1, g["nlon"] - 1)),
                             ((0, 512), (0, g["nlon"] - 1))):
        la, lo = _node_deg(nodes, a, b)
        fla, flo = _node_deg(g, fa, fb)
        assert abs(la - fla) < 1e-9 and abs(lo - flo) < 1e-9
    # a cell centre lies halfway between its corner nodes
    for i, j in ((0, 0), (100, 300), (511, 511)):
        c = _node_deg(centres, i, j)
        p, q = _node_deg(nodes, i, j), _node_deg(nodes, i + 1, j + 1)
        assert abs(c[0] - 0.5 * (p[0] + q[0])) < 1e-9 and abs(c[1] - 0.5 * (p[1] + q[1])) < 1e-9


def test_node_of_inverts_the_node_formula_and_cell_of_floors_it():
    g = sim.learned(5).grid
    nodes, _ = L.footprint_grids(g, 512)
    rng = np.random.default_rng(0)
    for _ in range(50):
        i, j = rng.uniform(0, g["nlat"] - 1), rng.uniform(0, g["nlon"] - 1)
        ri, rj = L.node_of(g, *_node_deg(g, i, j))
        assert abs(ri - i) < 1e-6 and abs(rj - j) < 1e-6
        ci, cj = rng.uniform(0, 512), rng.uniform(0, 512)
        assert L.cell_of(nodes, *_node_deg(nodes, ci, cj)) == (math.floor(ci), math.floor(cj))


def test_degrees_per_metre_matches_the_radii():
    for lat in (0.0, 30.0, 60.0, 85.0):
        dlat, dlon = L.degrees_per_metre(lat)
        e2 = F * (2.0 - F)
        w = math.sqrt(1.0 - e2 * math.sin(math.radians(lat)) ** 2)
        assert abs(dlat * math.radians(1.0) * A * (1.0 - e2) / w ** 3 - 1.0) < 1e-12
        assert abs(dlon * math.radians(1.0) * A / w * math.cos(math.radians(lat)) - 1.0) < 1e-12
    # one degree of latitude is ~110.6 km at the equator and ~111.7 km at the poles
    assert abs(1.0 / L.degrees_per_metre(0.0)[0] - 110574.0) < 2.0
    assert abs(1.0 / L.degrees_per_metre(89.999)[0] - 111694.0) < 2.0


def test_target_map_and_crops_keep_the_emitter():
    import torch
    t = L.target_map(64, 20, 33)
    assert t[20, 33] == 1.0 and t.max() == 1.0
    assert abs(t[21, 33] - math.exp(-0.5)) < 1e-12 and t[20, 40] == 0.0  # cut below 1e-3
    maps = torch.from_numpy(np.random.default_rng(1).standard_normal((3, 200, 200)).astype(np.float32))
    rng = np.random.default_rng(2)
    ci, cj = 150, 7
    xs, ts = training.make_crops(maps, ci, cj, 64, rng)
    assert len(xs) == len(ts) == 3
    full = L.target_map(200, ci, cj)
    for k, (x, tk) in enumerate(zip(xs, ts)):
        assert tuple(x.shape) == (3, 64, 64) and tk.shape == (64, 64)
        # each crop is a window of the maps, and its target the same window of the full target
        hits = [(i0, j0) for i0 in range(137) for j0 in range(137)
                if torch.equal(maps[:, i0:i0 + 64, j0:j0 + 64], x)]
        assert len(hits) == 1
        i0, j0 = hits[0]
        assert np.array_equal(tk, full[i0:i0 + 64, j0:j0 + 64])
        if k < 2:  # the crops around the emitter hold its cell
            assert 0 <= ci - i0 < 64 and 0 <= cj - j0 < 64 and tk[ci - i0, cj - j0] == 1.0


def test_unsure_search_criteria():
    """The fallback's unsure-search rule: the best proposal's logit under
    min_logit, or the best region's maximum less than min_region_gap
    (relative) above the runner-up's; either criterion can be switched off."""
    import types

    import torch

    from paper_2508_06672_gb300.learned import LearnedSearch

    s = types.SimpleNamespace(torch=torch, min_logit=3.6, min_region_gap=0.2,
                              geo=types.SimpleNamespace(stream=None))
    costs = torch.zeros((3, 5, 5))
    costs[0, 2, 2], costs[1, 1, 1], costs[2, 3, 3] = 10.0, 7.0, 1.0
    peaks = [{"value": 5.0}, {"value": 4.0}, {"value": 1.0}]
    assert not LearnedSearch.unsure(s, peaks, costs)            # margin 0.3, logit 5
    costs[1, 1, 1] = 8.5
    assert LearnedSearch.unsure(s, peaks, costs)                # margin 0.15 < 0.2
    s.min_region_gap = None
    assert not LearnedSearch.unsure(s, peaks, costs)
    assert LearnedSearch.unsure(s, [{"value": 3.5}, {"value": 2.0}], costs[:2])  # logit 3.5 < 3.6
    s.min_logit = None
    assert not LearnedSearch.unsure(s, [{"value": 3.5}], costs[:1])
