"""Pins of the oracle's refinement lattice (oracle.refine_grid): the dense
re-evaluation around the coarse maximum that Algorithm 1's search is repeated
on. The lattice must be centred exactly on the coarse node, its neighbouring
nodes must lie spacing_m apart on the WGS-84 ellipsoid (checked with the
simulator's independent numpy conversion, not the oracle's), and it must hold
round(window / spacing) nodes on each side, rounded half away from zero."""
import math

import numpy as np
import pytest

import oracle
import sim


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


COARSE = dict(lat0_deg=47.3, lon0_deg=-121.7, dlat_m=400.0, dlon_m=400.0, nlat=31, nlon=45)


def _node_deg(grid, i, j):
    lat, lon = oracle.grid_node(grid, i, j)
    return math.degrees(lat), math.degrees(lon)


@pytest.mark.parametrize("index", [0, 7 * 45 + 30, 31 * 45 - 1])
def test_centre_is_the_coarse_node_exactly(index):
    rg = oracle.refine_grid(COARSE, index, 25.0, 500.0)
    lat, lon = oracle.grid_node(COARSE, index // COARSE["nlon"], index % COARSE["nlon"])
    assert rg["lat0_deg"] == math.degrees(lat) and rg["lon0_deg"] == math.degrees(lon)
    half = rg["nlat"] // 2
    # the lattice's own middle node is its centre, bit for bit
    assert _node_deg(rg, half, half) == (rg["lat0_deg"], rg["lon0_deg"])
    # rows and columns are not swapped: the coarse node's row is its latitude
    i, j = divmod(index, COARSE["nlon"])
    lat_i, lon_j = _node_deg(COARSE, i, j)
    assert rg["lat0_deg"] == lat_i and rg["lon0_deg"] == lon_j


@pytest.mark.parametrize("spacing", [10.0, 25.0, 100.0])
@pytest.mark.parametrize("lat0", [0.0, 18.0, -63.5])
def test_neighbours_are_spacing_metres_apart_on_the_ellipsoid(spacing, lat0):
    coarse = dict(COARSE, lat0_deg=lat0)
    rg = oracle.refine_grid(coarse, 15 * 45 + 22, spacing, 8 * spacing)
    h = rg["nlat"] // 2
    # the two neighbours on either side of the centre, along each axis:
    # half their chord is the spacing (the first-order change of the radii of
    # curvature cancels between the two sides)
    for (a, b) in (((h - 1, h), (h + 1, h)), ((h, h - 1), (h, h + 1))):
        pa = sim.geodetic_to_ecef(*_node_deg(rg, *a))
        pb = sim.geodetic_to_ecef(*_node_deg(rg, *b))
        d = 0.5 * float(np.linalg.norm(pa - pb))
        assert abs(d / spacing - 1.0) < 1e-7, (a, b, d)
    # and the spacing is in metres, not degrees: one step is a tiny angle
    assert rg["dlat_m"] == spacing and rg["dlon_m"] == spacing


@pytest.mark.parametrize("window,spacing,half", [
    (1000.0, 100.0, 10),
    (240.0, 100.0, 2),    # 2.4 -> 2
    (250.0, 100.0, 3),    # 2.5: half away from zero (half to even would give 2)
    (260.0, 100.0, 3),    # 2.6: rounding gives 3 where flooring would give 2
    (350.0, 100.0, 4),    # 3.5 -> 4 (half to even would also give 4)
    (199.0, 25.0, 8),     # 7.96 -> 8, floor 7
    (25.0, 25.0, 1),
])
def test_half_width_rounds_half_away_from_zero(window, spacing, half):
    rg = oracle.refine_grid(COARSE, 0, spacing, window)
    assert rg["nlat"] == rg["nlon"] == 2 * half + 1


def test_extent_spans_the_window():
    rg = oracle.refine_grid(COARSE, 10 * 45 + 10, 50.0, 1000.0)
    h = rg["nlat"] // 2
    p0 = sim.geodetic_to_ecef(*_node_deg(rg, 0, h))
    p1 = sim.geodetic_to_ecef(*_node_deg(rg, 2 * h, h))
    assert abs(np.linalg.norm(p1 - p0) / 2000.0 - 1.0) < 1e-6
