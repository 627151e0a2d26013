"""Threshold detection of emitters (Algorithm 1, last step) on the device:
dg_detect against oracle.detect, on the same surfaces, index for index."""
import math

import numpy as np
import pytest

import oracle
import sim
from gpu_common import gpu_surface, package, torch_cuda
from oracle_pins import _bumps

pytestmark = pytest.mark.gpu


def _ctx(shape, prec="fp32", row0=0, nrows=0, lat0=48.0, lon0=11.0):
    torch_cuda()
    P = package()
    grid = dict(lat0_deg=lat0, lon0_deg=lon0, dlat_m=500.0, dlon_m=700.0, nlat=shape[0], nlon=shape[1])
    eph = sim.Formation().ephemerides(1)
    return P.Geolocator(grid, eph, 5e6, 1575.42e6, prec=prec, row0=row0, nrows=nrows), grid


def _dev(g, v):
    torch = g.torch
    return torch.from_numpy(np.ascontiguousarray(v)).to(device=g.device, dtype=g.dtype)


def _as_ctx_precision(v, prec):
    return v.astype(np.float32).astype(np.float64) if prec == "fp32" else v


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_detect_known_bumps(prec):
    centres, amps = [(5, 40), (30, 7), (33, 44), (0, 0)], [5.0, 3.0, 1.0, 2.0]
    v = _as_ctx_precision(_bumps((41, 53), centres, amps), prec)
    g, grid = _ctx((41, 53), prec)
    for thr, rad, mp in ((0.5, 3, 16), (2.5, 3, 16), (0.5, 3, 1), (0.5, 0, 2048)):
        want = oracle.detect(v, thr, rad, max_peaks=mp)
        got = g.detect(_dev(g, v), thr, radius=rad, max_peaks=mp)
        assert [p["index"] for p in got] == list(want)
        for p in got:
            assert p["value"] == v.flat[p["index"]]
            assert (p["i"], p["j"]) == divmod(p["index"], 53)
            lat, lon = oracle.grid_node(grid, p["i"], p["j"])
            assert abs(math.radians(p["lat_deg"]) - lat) < 1e-12
            assert abs(math.radians(p["lon_deg"]) - lon) < 1e-12
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,r", [((64, 64), 1), ((37, 129), 2), ((300, 301), 3), ((1, 700), 4)])
def test_detect_ties_bit_exact(prec, shape, r):
    """Integer-valued random surfaces (many equal values, plateaus): the same
    peaks in the same order as the oracle."""
    rng = np.random.default_rng(shape[0] * 1000 + shape[1] + r)
    v = rng.integers(0, 12, size=shape).astype(np.float64)
    g, _ = _ctx(shape, prec)
    thr = 7.0
    want = oracle.detect(v, thr, r, max_peaks=2048)
    assert 0 < len(want) <= 2048
    got = g.detect(_dev(g, v), thr, radius=r, max_peaks=2048)
    assert [p["index"] for p in got] == list(want)
    g.close()


def test_detect_relative_threshold_and_shard():
    """relative=1 scales the threshold by the surface maximum; a row shard
    reports global rows and looks only within its own rows."""
    v = _bumps((40, 30), [(3, 3), (20, 15), (36, 25)], [1.0, 4.0, 2.0])
    g, _ = _ctx((60, 30), "fp64", row0=10, nrows=40)
    got = g.detect(_dev(g, v), 0.4, relative=True, radius=3)
    want = oracle.detect(v, 0.4 * v.max(), 3)
    assert [p["index"] for p in got] == list(want)
    assert [p["i"] for p in got] == [10 + int(k) // 30 for k in want]
    g.close()


def test_detect_errors():
    P = package()
    g, _ = _ctx((50, 50), "fp32")
    v = _dev(g, np.zeros((50, 50)))
    with pytest.raises(P.DGError):
        g.detect(v, 0.0, radius=65)
    with pytest.raises(P.DGError):
        g.detect(v, 0.0, max_peaks=0)
    with pytest.raises(P.DGError):
        g.detect(v, float("nan"))
    with pytest.raises(P.DGError):
        g.detect(v, -1.0, radius=0)  # 2500 equal peaks: more than the sort holds at any threshold
    # nothing above the threshold: an empty list, not an error
    assert g.detect(v, 1.0, radius=2) == []
    nan = _dev(g, np.full((50, 50), np.nan))
    with pytest.raises(P.DGError):
        g.detect(nan, 0.5, relative=True)
    # the context stays usable after the rejected calls
    w = _dev(g, _bumps((50, 50), [(25, 25)], [1.0]))
    assert [p["index"] for p in g.detect(w, 0.5, radius=3)] == [25 * 50 + 25]
    g.close()


@pytest.fixture(scope="module")
def crowded():
    return sim.crowded()


@pytest.fixture(scope="module")
def crowded_oracle(crowded):
    return oracle.cost_surface(*oracle.scene_args(crowded), acc_mode=1).reshape(121, 121)


def _near(nodes, peaks, tol=1):
    return all(any(abs(p["i"] - i) <= tol and abs(p["j"] - j) <= tol for p in peaks) for i, j in nodes)


@pytest.mark.parametrize("opts", [dict(prec="fp32"),
                                  dict(prec="fp32", algo="cdft", chunk=1024, contract="fp16x3")],
                         ids=["direct", "cdft_fp16x3"])
def test_detect_crowded_scene(crowded, crowded_oracle, opts):
    """Three simultaneous emitters (two noise, one chirp, one 3 dB weaker):
    the magnitude-accumulated surface thresholded at half its maximum gives
    exactly three detections, one on each emitter's node, on the device as in
    the oracle; the device detector on the oracle's surface reproduces the
    oracle's detections exactly."""
    g, c = gpu_surface(crowded, acc="mag", **opts)
    ref = crowded_oracle
    want = oracle.detect(ref, 0.5 * ref.max(), 3)
    assert [divmod(int(k), 121) for k in want] == sorted(crowded.emitter_nodes, key=lambda n: -ref[n])
    cost = g.cost_surface()
    got = g.detect(cost, 0.5, relative=True, radius=3)
    assert len(got) == 3 and _near(crowded.emitter_nodes, got, tol=0)
    exact = g.detect(_dev(g, ref), 0.5 * float(np.float32(ref.max())), radius=3)
    assert [p["index"] for p in exact] == list(oracle.detect(ref.astype(np.float32).astype(np.float64),
                                                             0.5 * float(np.float32(ref.max())), 3))
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("max_peaks", [1, 8, 300])
def test_detect_more_peaks_than_the_sort_holds(prec, max_peaks):
    """A noisy surface with ~10k local maxima (more than the 2048 the device
    sort holds) and a wide plateau above most of them: the threshold is
    raised until the sort holds every peak that passes, and the result is
    the oracle's, index for index."""
    rng = np.random.default_rng(11 + max_peaks)
    v = rng.uniform(0.0, 1.0, size=(300, 301))
    v[100:160, 50:200] = 0.9995          # one plateau: one peak, its lowest index
    v[20, 20] = 2.0
    v = _as_ctx_precision(v, prec)
    g, _ = _ctx(v.shape, prec)
    want = oracle.detect(v, -1.0, 1, max_peaks=max_peaks)
    assert len(oracle.detect(v, -1.0, 1, max_peaks=20000)) > 2048
    got = g.detect(_dev(g, v), -1.0, radius=1, max_peaks=max_peaks)
    assert [p["index"] for p in got] == list(want) and len(got) == max_peaks
    g.close()
