"""The learned-proposal workload's geometry (CPU).

With both receivers in one orbit plane, TDOA and FDOA are symmetric about
the plane through the Earth's centre and the two receivers, so an emitter's
mirror image across it is an equally good candidate. The workload places its
2000 km footprint wholly on one side of that plane (formation near its
orbit's northern apex, footprint 1200 km toward the equator), and the
emitter at least 60 km inside the footprint's edges."""
import math

import numpy as np
import pytest

import sim
from paper_2508_06672_gb300 import learned as L

A, F = 6378137.0, 1.0 / 298.257223563


def _ecef(grid, i, j):
    e2 = F * (2.0 - F)
    lat0 = math.radians(grid["lat0_deg"])
    w = math.sqrt(1.0 - e2 * math.sin(lat0) ** 2)
    m, n = A * (1.0 - e2) / w ** 3, A / w
    lat = lat0 + (i - 0.5 * (grid["nlat"] - 1)) * grid["dlat_m"] / m
    lon = math.radians(grid["lon0_deg"]) + (j - 0.5 * (grid["nlon"] - 1)) * grid["dlon_m"] / (n * math.cos(lat0))
    nn = A / math.sqrt(1.0 - e2 * math.sin(lat) ** 2)
    return np.array([nn * math.cos(lat) * math.cos(lon), nn * math.cos(lat) * math.sin(lon),
                     nn * (1.0 - e2) * math.sin(lat)])


@pytest.mark.parametrize("seed", [5, 1000, 100005, 200000, 300000])
def test_footprint_on_one_side_and_emitter_inside(seed):
    s = sim.learned(seed)
    g = s.grid
    n = g["nlat"]
    assert g["nlon"] == n == 4001
    edge = [(a, b) for a in (0, n // 2, n - 1) for b in range(0, n, 250)]
    edge += [(b, a) for a, b in edge]
    eph = np.asarray(s.ephem, dtype=np.float64).reshape(-1, 12)
    sides = []
    for k in (0, eph.shape[0] - 1):
        p1, p2 = eph[k, 0:3], eph[k, 6:9]
        nrm = np.cross(p1, p2)
        nrm /= np.linalg.norm(nrm)
        d = np.array([nrm @ _ecef(g, i, j) for i, j in edge])
        assert np.all(np.sign(d) == np.sign(d[0]))
        assert np.abs(d).min() > 50e3  # metres from the plane
        sides.append(np.sign(d[0]))
    assert sides[0] == sides[1]
    ci, cj = L.node_of(g, s.emitter_lat_deg, s.emitter_lon_deg)
    margin = 60e3 / g["dlat_m"] - 1.0
    assert margin <= ci <= n - 1 - margin and margin <= cj <= n - 1 - margin
