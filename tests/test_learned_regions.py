"""Regions of the learned search are made of nodes of the full search's grid.

A grid's node spacing is given in metres and turned into degrees with the
WGS-84 meridian and prime-vertical radii at the grid's own centre latitude
(row i at lat0 + (i - (n - 1) / 2) dlat_m / M(lat0), column j likewise with
N(lat0) cos(lat0)). Over a 2000 km footprint those radii change by up to
~12 % in longitude, so a region centred 800 km from the footprint's centre
must take other spacings in metres to land on the full grid's nodes. CPU
only: the node positions are computed here from the definition above."""
import math

import sim
from paper_2508_06672_gb300 import learned as L

A, F = 6378137.0, 1.0 / 298.257223563


def _node(grid, i, j):
    e2 = F * (2.0 - F)
    lat0 = math.radians(grid["lat0_deg"])
    w = math.sqrt(1.0 - e2 * math.sin(lat0) ** 2)
    m, n = A * (1.0 - e2) / w ** 3, A / w
    return (lat0 + (i - 0.5 * (grid["nlat"] - 1)) * grid["dlat_m"] / m,
            math.radians(grid["lon0_deg"]) + (j - 0.5 * (grid["nlon"] - 1)) * grid["dlon_m"] / (n * math.cos(lat0)))


class _Search:
    region_grid = L.LearnedSearch.region_grid

    def __init__(self, grid, half):
        self.grid, self.half = grid, half


def test_region_nodes_are_full_grid_nodes():
    grid = sim.learned(5).grid
    s = _Search(grid, 50)
    for dlat, dlon in ((7.0, -6.0), (-8.0, 9.0), (0.0, 0.0), (-9.3, -12.0)):
        r = s.region_grid(grid["lat0_deg"] + dlat, grid["lon0_deg"] + dlon)
        assert r["nlat"] == r["nlon"] == 101
        ci, cj = L.node_of(grid, r["lat0_deg"], r["lon0_deg"])
        assert abs(ci - round(ci)) < 1e-6 and abs(cj - round(cj)) < 1e-6
        ci, cj = round(ci), round(cj)
        for a in (0, 37, 50, 100):
            for b in (0, 50, 91, 100):
                la, lo = _node(r, a, b)
                fa, fo = _node(grid, ci + a - 50, cj + b - 50)
                assert abs(la - fa) * A < 1e-6 and abs(lo - fo) * A < 1e-6
    # away from the centre latitude the east-west spacing in metres differs
    far = s.region_grid(grid["lat0_deg"] + 7.0, grid["lon0_deg"])
    assert abs(far["dlon_m"] / grid["dlon_m"] - 1.0) > 0.05
