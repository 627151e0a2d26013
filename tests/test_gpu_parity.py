"""CUDA library (through the C ABI) against the CPU oracle, element by element.

Tolerances:
  * integer lags (Eq. 9): bit-exact; argmax indices: bit-exact wherever the
    oracle's two largest values differ by more than twice the error bound,
    otherwise the device's maximum must be within that bound of the oracle's;
  * FP64 surfaces: relative 1e-9;
  * FP32 surfaces: relative 1e-4 per point (the bound the FP32 path is held
    to); for surfaces of only a few snapshots a floor of 1% of the surface
    mean is added to the denominator, because FP32 rounding error in C is
    absolute (~eps N |y|^2) and |C_k| of single snapshots can be arbitrarily
    close to zero.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import sim
from gpu_common import (assert_argmax_consistent, assert_global_argmax, gpu_surface, lag_boundary_mask,
                        oracle_surface, package, rel_err, torch_cuda)

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
FP64_TOL = 1e-9


# ------------------------------------------------------------ a1: grid -> ECEF
@pytest.mark.parametrize("rows", [None, (3, 11)])
def test_grid_ecef(rows):
    torch = torch_cuda()
    P = package()
    grid = dict(lat0_deg=-33.3, lon0_deg=151.2, dlat_m=850.0, dlon_m=1200.0, nlat=17, nlon=23)
    r0, nr = (0, 0) if rows is None else (rows[0], rows[1] - rows[0])
    g = P.Geolocator(grid, np.zeros((1, 12)) + 7e6, 5e6, 1575.42e6, row0=r0, nrows=nr)
    xyz = g.grid_ecef().cpu().numpy()
    ref = oracle.grid_ecef(grid).reshape(17, 23, 3)
    if rows is not None:
        ref = ref[rows[0]:rows[1]]
    ref = ref.reshape(-1, 3).T
    assert np.max(np.abs(xyz - ref)) < 1e-6
    g.close()


# ------------------------------------------------------- a2/a3: the geometry
def test_step_geometry_lags_exact():
    torch_cuda()
    s = sim.mid(grid_n=(61, 53), k_steps=4, n_samples=64)
    for delay in ("integer", "lagrange4"):
        g, _ = gpu_surface(s, delay=delay)
        dm = 0 if delay == "integer" else 1
        idx = np.arange(s.G)
        _, geom = oracle.cost_points(*oracle.scene_args(s), idx=idx, want_geom=True, delay_mode=dm)
        near = lag_boundary_mask(s, idx, dm)
        for k in range(s.k_steps):
            lag, D, nu = (t.cpu().numpy() for t in g.step_geometry(k))
            Dr, nur = geom[:, k, 2], geom[:, k, 3]
            # Eq. 9: round half away from zero; fractional mode: floor
            Lr = np.sign(Dr) * np.floor(np.abs(Dr) + 0.5) if dm == 0 else np.floor(Dr)
            ok = ~near
            assert np.array_equal(lag[ok], Lr[ok].astype(np.int32)), (delay, k)
            assert np.all(np.abs(lag[~ok] - Lr[~ok]) <= 1)
            assert np.max(np.abs(D - Dr)) < 1e-9
            assert np.max(np.abs(nu - nur)) < 1e-15
        assert near.sum() <= max(1, s.G // 1000)
        g.close()


# ------------------------------------------- workload 1 (tiny): full grid, FP64
def test_tiny_workload_fp64_full_grid():
    s = sim.tiny()
    g, c = gpu_surface(s, prec="fp64")
    ref = oracle_surface(s)
    assert rel_err(c, ref) < FP64_TOL
    assert_argmax_consistent(c, ref, FP64_TOL)
    g.close()


def test_tiny_workload_fp32_matches_fp64_oracle():
    s = sim.tiny()
    g, c = gpu_surface(s, prec="fp32")
    ref = oracle_surface(s)
    # one snapshot: values near zero exist, so the floor applies
    assert rel_err(c, ref, floor_frac=0.01) < FP32_TOL
    g.close()


# ------------------------------------- workload 2 (mid): sub-grid at full K, N
def test_mid_workload_subgrid_fp32():
    s = sim.mid(grid_n=(49, 41))
    g, c = gpu_surface(s)
    ref = oracle_surface(s)
    idx = np.arange(s.G)
    ok = ~lag_boundary_mask(s, idx)
    assert rel_err(c.ravel()[ok], ref.ravel()[ok]) < FP32_TOL
    am = assert_argmax_consistent(c, ref, FP32_TOL)
    srt = np.sort(ref.ravel())[::-1]
    # The noisy chirp leaves a cross-track ridge (one snapshot resolves
    # Doppler to ~190 Hz): the maximum lies on it near the emitter, and the
    # emitter's own node is within 10% of the maximum.
    centre = (s.grid["nlat"] // 2) * s.grid["nlon"] + s.grid["nlon"] // 2
    di, dj = np.subtract(divmod(am, s.grid["nlon"]), divmod(centre, s.grid["nlon"]))
    assert abs(di) <= 10 and abs(dj) <= 10
    assert ref.ravel()[centre] > 0.9 * srt[0]
    g.close()


@pytest.mark.parametrize("delay,dm", [("integer", 0), ("lagrange4", 1)])
def test_mid_geometry_noise_free_peaks_at_emitter(delay, dm):
    """Noise-free 5 MHz noise emitter on the mid-size geometry, full K and N:
    oracle and device both put the maximum on the emitter's node (Sec. IV-B:
    the accumulated peak sits at the true position). (A chirp filling 80% of
    the band is not used here: the 4-tap interpolator's error near the band
    edge favours nodes with a near-integer delay.)"""
    s = sim.mid(grid_n=(21, 21), snr_db=None, waveform="noise", bw_hz=5e6)
    g, c = gpu_surface(s, delay=delay)
    ref = oracle_surface(s, dm)
    centre = 10 * 21 + 10
    assert oracle.argmax(ref) == centre
    # integer lags: the emitter's node leads its neighbour by only ~2.6e-5 of
    # the maximum (a near-tie at the FP32 bound); Lagrange4: by ~4.4e-4
    assert_argmax_consistent(c, ref, FP32_TOL, near_tie=(dm == 0))
    assert rel_err(c, ref) < FP32_TOL
    g.close()


# ---------------------- ragged tiles, odd N, both delay and accumulation modes
@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
@pytest.mark.parametrize("delay", ["integer", "lagrange4"])
@pytest.mark.parametrize("acc", ["power", "mag"])
def test_small_scenes_all_modes(fmt, delay, acc):
    s = sim.make_scene(seed=21, fs_hz=12.5e6, n_samples=3001, k_steps=3, fmt=fmt, waveform="chirp",
                       snr_db=-3.0, grid_n=(37, 45), grid_spacing_m=150.0)
    dm, am = (0 if delay == "integer" else 1), (0 if acc == "power" else 1)
    for prec, tol, floor in (("fp32", FP32_TOL, 0.01), ("fp64", FP64_TOL, 0.0)):
        g, c = gpu_surface(s, delay=delay, acc=acc, prec=prec)
        ref = oracle_surface(s, dm, am)
        idx = np.arange(s.G)
        ok = ~lag_boundary_mask(s, idx, dm)
        assert rel_err(c.ravel()[ok], ref.ravel()[ok], floor) < tol, (prec, fmt, delay, acc)
        g.close()


# -------------------------------------------------------------- edge cases
def test_single_node_single_sample_and_lags_beyond_capture():
    torch = torch_cuda()
    P = package()
    # one candidate, one sample
    s = sim.make_scene(seed=5, fs_hz=5e6, n_samples=1, k_steps=2, fmt="c64", waveform="noise",
                       snr_db=0.0, grid_n=1, grid_spacing_m=100.0)
    g, c = gpu_surface(s, prec="fp64")
    assert rel_err(c, oracle_surface(s)) < FP64_TOL
    g.close()
    # captures shorter than every lag: no overlap, the surface is exactly zero
    s = sim.make_scene(seed=6, fs_hz=20e6, n_samples=8, k_steps=1, fmt="ci16", waveform="noise",
                       snr_db=0.0, grid_n=(5, 7), grid_spacing_m=20000.0)
    ref = oracle_surface(s)
    g, c = gpu_surface(s)
    assert np.array_equal(c == 0, ref == 0)
    assert rel_err(c[ref > 0], ref[ref > 0], 0.01) < FP32_TOL if np.any(ref > 0) else True
    g.close()


@pytest.mark.parametrize("spacing,shape", [(6000.0, (70, 33)), (20000.0, (70, 40))])
def test_wide_lag_spans(spacing, shape):
    """A tile whose lag span nearly fills the shared-memory window runs with
    shorter chunks (6 km grid); one whose span exceeds it reads y2 from global
    memory (20 km grid). Same results as the oracle either way."""
    torch_cuda()
    s = sim.make_scene(seed=8, fs_hz=20e6, n_samples=6000, k_steps=2, fmt="ci8", waveform="noise",
                       snr_db=-5.0, grid_n=shape, grid_spacing_m=spacing, bw_hz=18e6)
    idx = np.arange(s.G)
    _, geom = oracle.cost_points(*oracle.scene_args(s), idx=idx, want_geom=True)
    tile_span = np.ptp(geom[:, 0, 2].reshape(shape)[:64, :32])
    assert tile_span > (4000 if spacing > 10000 else 2000)
    for delay, dm in (("integer", 0), ("lagrange4", 1)):
        g, c = gpu_surface(s, delay=delay)
        ref = oracle_surface(s, dm)
        ok = ~lag_boundary_mask(s, idx, dm)
        assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
        g.close()


def test_row_shards_concatenate_bit_exactly():
    s = sim.make_scene(seed=9, fs_hz=12.5e6, n_samples=2048, k_steps=2, fmt="ci16", waveform="chirp",
                       snr_db=-5.0, grid_n=(77, 41), grid_spacing_m=120.0)
    g, full = gpu_surface(s)
    g.close()
    parts = []
    for r0, r1 in ((0, 30), (30, 77)):
        g, c = gpu_surface(s, row0=r0, nrows=r1 - r0)
        parts.append(c)
        g.close()
    assert np.array_equal(np.concatenate(parts), full)


def test_mixed_formats_and_lengths_per_snapshot():
    torch = torch_cuda()
    P = package()
    a = sim.make_scene(seed=12, fs_hz=12.5e6, n_samples=1500, k_steps=2, fmt="ci16", waveform="chirp",
                       snr_db=-3.0, grid_n=(9, 11), grid_spacing_m=200.0)
    b = sim.make_scene(seed=12, fs_hz=12.5e6, n_samples=2501, k_steps=2, fmt="c64", waveform="chirp",
                       snr_db=-3.0, grid_n=(9, 11), grid_spacing_m=200.0)
    g = P.Geolocator(a.grid, a.ephem, a.fs_hz, a.fc_hz, prec="fp64")
    g.load_capture(0, "ci16", torch.from_numpy(a.y1[0]).cuda(), torch.from_numpy(a.y2[0]).cuda())
    g.load_capture(1, "c64", torch.from_numpy(b.y1[1]).cuda(), torch.from_numpy(b.y2[1]).cuda())
    c = g.cost_surface().cpu().numpy()
    ref = sum(oracle.cost_surface(a.grid, a.ephem[k:k + 1], a.fs_hz, a.fc_hz, s.y1[k:k + 1], s.y2[k:k + 1])
              for k, s in ((0, a), (1, b)))
    assert rel_err(c, ref) < FP64_TOL
    g.close()


# --------------------------------------------------- a8: argmax and refinement
def test_argmax_and_refine_match_oracle():
    s = sim.tiny(grid_n=41)
    g, _ = gpu_surface(s, prec="fp64")
    torch = torch_cuda()
    cost = g.cost_surface()
    fix = g.argmax_refine(cost, 100.0, 1000.0)
    ref = oracle_surface(s)
    am = oracle.argmax(ref)
    assert fix["index"] == am and (fix["i"], fix["j"]) == divmod(am, s.grid["nlon"])
    lat, lon = oracle.grid_node(s.grid, fix["i"], fix["j"])
    assert abs(fix["lat_deg"] - np.degrees(lat)) < 1e-12 and abs(fix["lon_deg"] - np.degrees(lon)) < 1e-12
    lg = oracle.refine_grid(s.grid, am, 100.0, 1000.0)
    lref = oracle.cost_surface(lg, s.ephem, s.fs_hz, s.fc_hz, s.y1, s.y2)
    assert fix["refine_n"] == lg["nlat"] == 21
    lam = oracle.argmax(lref)
    assert (fix["ri"], fix["rj"]) == divmod(lam, lg["nlon"])
    assert abs(fix["refined_cost"] / lref.ravel()[lam] - 1) < FP64_TOL
    # the parabolic sub-node estimate around the refined maximum, from the
    # oracle's refinement surface (FP64 on both sides: offsets agree to 1e-4 node)
    ri, rj = divmod(lam, lg["nlon"])
    di, dj = oracle.subcell(lref.reshape(lg["nlat"], lg["nlon"]), ri, rj)
    dlat, dlon = oracle.grid_step_rad(lg)
    assert abs(fix["sub_lat_deg"] - fix["refined_lat_deg"] - np.degrees(di * dlat)) <= 1e-4 * np.degrees(dlat)
    assert abs(fix["sub_lon_deg"] - fix["refined_lon_deg"] - np.degrees(dj * dlon)) <= 1e-4 * np.degrees(dlon)
    assert abs(di) <= 0.5 and abs(dj) <= 0.5 and (di, dj) != (0.0, 0.0)
    # no refinement requested: around the grid maximum
    f0 = g.argmax_refine(cost)
    assert f0["refine_n"] == 0 and f0["index"] == am
    di, dj = oracle.subcell(ref.reshape(s.grid["nlat"], s.grid["nlon"]), *divmod(am, s.grid["nlon"]))
    dlat, dlon = oracle.grid_step_rad(s.grid)
    assert abs(f0["sub_lat_deg"] - f0["lat_deg"] - np.degrees(di * dlat)) <= 1e-4 * np.degrees(dlat)
    assert abs(f0["sub_lon_deg"] - f0["lon_deg"] - np.degrees(dj * dlon)) <= 1e-4 * np.degrees(dlon)
    g.close()


def test_argmax_ties_and_nan_on_device():
    torch = torch_cuda()
    s = sim.tiny(grid_n=(3, 5), n_samples=64)
    P = package()
    g = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz)
    v = torch.tensor([1.0, 7.0, float("nan"), 7.0, 2.0] * 3, dtype=torch.float32, device="cuda")
    assert g.argmax_refine(v)["index"] == 1
    v = torch.full((15,), float("nan"), dtype=torch.float32, device="cuda")
    with pytest.raises(P.DGError):
        g.argmax_refine(v)
    g.close()


# --------------------------------------------- workloads at full size, sampled
def _sampled_check(s, c, npts, seed, floor=0.0):
    """Pointwise bound on random nodes, then the complete argmax check over
    every node that can hold the oracle's maximum under that bound."""
    rng = np.random.default_rng(seed)
    idx = np.unique(rng.integers(0, s.G, npts))
    ref = oracle.cost_points(*oracle.scene_args(s), idx=idx)
    ok = ~lag_boundary_mask(s, idx)
    assert rel_err(c.ravel()[idx][ok], ref[ok], floor) < FP32_TOL
    return assert_global_argmax(s, c, FP32_TOL)


def test_mid_workload_full_size_sampled():
    s = sim.mid()
    g, c = gpu_surface(s)
    am = _sampled_check(s, c, 48, 2)
    di, dj = np.subtract(divmod(am, s.grid["nlon"]), (s.grid["nlat"] // 2, s.grid["nlon"] // 2))
    assert abs(di) <= 10 and abs(dj) <= 10  # on the ridge through the emitter
    g.close()


def test_large_workload_full_size_sampled():
    s = sim.large()
    g, c = gpu_surface(s)
    _sampled_check(s, c, 16, 3)
    g.close()


# ------------------------------------------------------------- error paths
def test_error_paths_leave_context_usable():
    torch = torch_cuda()
    P = package()
    s = sim.tiny(grid_n=(5, 5), n_samples=256)
    g = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz)
    with pytest.raises(P.DGError) as e:
        g.cost_surface()
    assert e.value.status == P.DG_ESTATE
    y = torch.from_numpy(s.y1[0]).cuda()
    with pytest.raises(P.DGError) as e:
        P.dg_load_capture(g.ctx, 1, P.DG_IQ_C64, y.data_ptr(), y.data_ptr(), 256, 1)
    assert e.value.status == P.DG_EINVAL
    with pytest.raises(P.DGError) as e:
        P.dg_load_capture(g.ctx, 0, 9, y.data_ptr(), y.data_ptr(), 256, 1)
    assert e.value.status == P.DG_EINVAL
    g.load_captures(s.fmt, s.y1, s.y2)
    c = g.cost_surface()
    g.sync()
    assert rel_err(c.cpu().numpy(), oracle_surface(s), 0.01) < FP32_TOL
    g.close()


def test_fdoa_out_of_range_is_reported():
    torch = torch_cuda()
    P = package()
    s = sim.tiny(grid_n=(5, 5), n_samples=256)
    eph = s.ephem.copy()
    eph[:, 9:12] *= 1000.0  # receiver 2 at ~7600 km/s: FDOA beyond 0.2 fs
    pc = oracle.grid_ecef(s.grid)[12]
    assert abs(oracle.geometry(pc, eph[0], s.fs_hz, s.fc_hz)[3]) > 0.2
    g = P.Geolocator(s.grid, eph, s.fs_hz, s.fc_hz)
    g.load_captures(s.fmt, s.y1, s.y2)
    g.cost_surface()
    with pytest.raises(P.DGError) as e:
        g.sync()
    assert e.value.status == P.DG_EUNSUPPORTED
    g.sync()  # the error was reported once; the context is usable
    g.close()
