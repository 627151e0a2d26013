"""Chunked-DFT evaluation (DG_ALGO_CDFT) against the CPU oracle.

Same tolerances as the direct path: relative 1e-4 per point for FP32
(floor of 1% of the mean for surfaces of one to three snapshots). The bin
interpolation adds ~(pi M Delta)^2/8 < 1e-6 at these geometries."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import sim
from gpu_common import (assert_argmax_consistent, assert_global_argmax, gpu_surface, lag_boundary_mask, oracle_surface, package,
                        rel_err, torch_cuda)

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-4


@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
@pytest.mark.parametrize("acc", ["power", "mag"])
def test_cdft_small_scenes(fmt, acc):
    s = sim.make_scene(seed=21, fs_hz=12.5e6, n_samples=3001, k_steps=3, fmt=fmt, waveform="chirp",
                       snr_db=-3.0, grid_n=(37, 45), grid_spacing_m=150.0)
    am = 0 if acc == "power" else 1
    g, c = gpu_surface(s, algo="cdft", acc=acc)
    ref = oracle_surface(s, 0, am)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
    g.close()


@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
@pytest.mark.parametrize("contract", ["bf16", "fp16x3"])
def test_cdft_lag_tiles_match_row_tiles(fmt, contract):
    """Tensor-core tiles of 128 consecutive lags at one chunk (shared capture
    windows) and tiles of consecutive (lag, chunk) rows form the same lag
    products: the surfaces are bit-identical, and within the form's bound of
    the oracle. Five blocks of 128 lags (75 .. 707), a ragged last chunk, and
    y2 windows that run off the end of the capture."""
    s = sim.make_scene(seed=24, fs_hz=20e6, n_samples=5000, k_steps=2, fmt=fmt, waveform="noise",
                       snr_db=-3.0, grid_n=(45, 41), grid_spacing_m=2000.0, bw_hz=18e6)
    out = {}
    for tiles in ("rows", "lags"):
        g, c = gpu_surface(s, algo="cdft", contract=contract, chunk=1024, tiles=tiles)
        out[tiles] = c
        g.close()
    assert np.array_equal(out["rows"], out["lags"])
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    # BF16 keeps 8 significant bits of each lag product and DFT entry: the
    # power |C|^2 of a noise-like node then carries a relative error of std
    # ~2^-8, and the maximum over ~1800 nodes of two snapshots reaches
    # ~4 std; the split form is held to the FP32 bound
    tol = TC_TOL[contract] if contract.endswith("x3") else 3e-2
    assert rel_err(out["lags"].ravel()[ok], ref.ravel()[ok], 0.01) < tol


@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
def test_cdft_mixed_tiles_match_row_and_lag_tiles(fmt):
    """AUTO on snapshots of 391 and 390 lags (three whole blocks of 128 and a
    remainder of 7 and 6): lag tiles over the whole blocks, row tiles over the
    remaining lags. Every tile kind forms the same lag products, so the three
    surfaces are bit-identical, and within the bound of the oracle."""
    s = sim.make_scene(seed=24, fs_hz=20e6, n_samples=5000, k_steps=2, fmt=fmt, waveform="noise",
                       snr_db=-3.0, grid_n=(45, 41), grid_spacing_m=1300.0, bw_hz=18e6)
    D, _ = oracle.node_geometry(s.grid, s.ephem, s.fs_hz, s.fc_hz)
    nb = [int(np.ptp(np.sign(d) * np.floor(np.abs(d) + 0.5))) + 1 for d in D]
    assert all(0 < n % 128 < 64 and n >= 128 for n in nb), nb  # the case AUTO splits
    out = {}
    for tiles in ("auto", "rows", "lags"):
        g, c = gpu_surface(s, algo="cdft", contract="fp16x3", chunk=1024, tiles=tiles)
        out[tiles] = c
        g.close()
    assert np.array_equal(out["auto"], out["rows"]) and np.array_equal(out["auto"], out["lags"])
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(out["auto"].ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL


@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
@pytest.mark.parametrize("contract", ["bf16x3", "fp16x3", "bf16", "fp16"])
def test_cdft_hankel_tiles(fmt, contract):
    """Hankel tiles (256 lags at one chunk; the DFT regrouped onto y1 and y2
    read as a Hankel matrix from shared memory) against the oracle within the
    form's bound, and against row tiles within twice it: two tiles of 512
    lags over 75 .. 707 (a ragged last tile), a ragged last chunk, and y2
    windows that run off the end of the capture."""
    s = sim.make_scene(seed=24, fs_hz=20e6, n_samples=5000, k_steps=2, fmt=fmt, waveform="noise",
                       snr_db=-3.0, grid_n=(45, 41), grid_spacing_m=2000.0, bw_hz=18e6)
    out = {}
    for tiles in ("rows", "hankel"):
        g, c = gpu_surface(s, algo="cdft", contract=contract, chunk=1024, tiles=tiles)
        out[tiles] = c
        g.close()
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    tol = TC_TOL[contract] if contract.endswith("x3") else 3e-2
    assert rel_err(out["hankel"].ravel()[ok], ref.ravel()[ok], 0.01) < tol
    assert rel_err(out["hankel"].ravel(), out["rows"].ravel(), 0.01) < 2 * tol


@pytest.mark.parametrize("chunk", [256, 512])
def test_cdft_hankel_shorter_chunks_and_auto(chunk):
    """Shorter chunks (fewer stages per tile), Hankel tiles against the
    oracle and AUTO beside them, and a grid of a few lags (row tiles)."""
    s = sim.make_scene(seed=27, fs_hz=12.5e6, n_samples=6000, k_steps=3, fmt="ci16", waveform="chirp",
                       snr_db=-3.0, grid_n=(33, 37), grid_spacing_m=3000.0)
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    for tiles in ("hankel", "auto"):
        g, c = gpu_surface(s, algo="cdft", contract="bf16x3", chunk=chunk, tiles=tiles)
        assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < TC_TOL["bf16x3"]
        g.close()
    # a grid of a few lags: AUTO picks row tiles there
    s2 = sim.make_scene(seed=28, fs_hz=12.5e6, n_samples=6000, k_steps=2, fmt="ci16", waveform="chirp",
                        snr_db=-3.0, grid_n=(9, 9), grid_spacing_m=50.0)
    g, c = gpu_surface(s2, algo="cdft", contract="bf16x3", chunk=chunk)
    ref2 = oracle_surface(s2)
    ok2 = ~lag_boundary_mask(s2, np.arange(s2.G))
    assert rel_err(c.ravel()[ok2], ref2.ravel()[ok2], 0.01) < TC_TOL["bf16x3"]
    g.close()


def test_cdft_auto_chunk():
    """chunk 0: each batch takes the longest power-of-two chunk up to 1024
    (few tiles here) whose length times the estimated bin spacing stays
    within the bound (with a 10 % margin); a grid with a wider FDOA span in
    cycles per sample (1000 km at 0.5 MHz) gets a shorter chunk. At 12.5 MHz
    the surface is held to the FP32 bound. At 0.5 MHz the FDOAs reach 6e-3
    cycles per sample, and their FP32 rounding limits every FP32 path: the
    direct evaluation measures 1.5e-4 on this scene (chunks of 128 and 512
    samples 1.2e-4 alike, so not the interpolation); that case is held to
    2e-4."""
    chunks = []
    for fs, spacing, tol in ((12.5e6, 100.0, FP32_TOL), (5e5, 25000.0, 2e-4)):
        s = sim.make_scene(seed=23, fs_hz=fs, n_samples=40000, k_steps=2, fmt="ci16", waveform="chirp",
                           snr_db=-3.0, grid_n=(41, 39), grid_spacing_m=spacing)
        g, c = gpu_surface(s, algo="cdft")
        lo, hi = g.cdft_chunks()
        assert lo & (lo - 1) == 0 and hi & (hi - 1) == 0 and 64 <= lo <= hi <= 1024
        ref = oracle_surface(s)
        ok = ~lag_boundary_mask(s, np.arange(s.G))
        r, d = ref.ravel()[ok], c.ravel()[ok]
        strong = r >= 0.1 * r.max()
        floored = np.max(np.abs(d - r) / (r + 0.01 * r.mean()))
        print(f"fs {fs:g}: chunk {hi}, floored error {floored:.3e}, "
              f"plain error on nodes >= 10% of the maximum {np.max(np.abs(d - r)[strong] / r[strong]):.3e}")
        assert rel_err(d, r, 0.01) < tol
        chunks.append(hi)
        g.close()
    assert chunks[1] < chunks[0]


@pytest.mark.parametrize("chunk", [2048, 3072])
def test_cdft_long_chunks_in_windows(chunk):
    """Chunks longer than the 1024-sample capture window: lag tiles stage each
    chunk in 1024-sample windows (the next prefetched while the current one's
    stages run). Their surfaces equal the row tiles' bit for bit (the same lag
    products, the same accumulation order) and the oracle's within the FP32
    bound, with a ragged last chunk and five blocks of 128 lags."""
    s = sim.make_scene(seed=28, fs_hz=20e6, n_samples=20001, k_steps=2, fmt="ci8", waveform="noise",
                       snr_db=-3.0, grid_n=(45, 41), grid_spacing_m=4000.0, bw_hz=18e6)
    out = {}
    for tiles in ("rows", "lags"):
        g, c = gpu_surface(s, algo="cdft", contract="fp16x3", chunk=chunk, tiles=tiles)
        out[tiles] = c
        g.close()
    assert np.array_equal(out["rows"], out["lags"])
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(out["lags"].ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL


def test_cdft_auto_chunk_above_the_window():
    """With many snapshots of long captures and a few hundred lags, the
    automatic chunk on the tensor cores grows past 1024 samples, to its cap
    of 2048, while the batch keeps enough lag tiles per SM (16 snapshots x
    about 1190 lags x 64 chunks); the surface stays within the FP32 bound of
    the oracle."""
    s = sim.make_scene(seed=29, fs_hz=20e6, n_samples=131072, k_steps=16, fmt="ci8", waveform="noise",
                       snr_db=-3.0, grid_n=(45, 41), grid_spacing_m=4000.0, bw_hz=18e6)
    g, c = gpu_surface(s, algo="cdft", contract="fp16x3")
    lo, hi = g.cdft_chunks()
    assert lo == hi == 2048, (lo, hi)
    g.close()
    rng = np.random.default_rng(3)
    idx = np.unique(rng.integers(0, s.G, 200))
    ref = oracle.cost_points(*oracle.scene_args(s), idx=idx)
    ok = ~lag_boundary_mask(s, idx)
    assert rel_err(c.ravel()[idx][ok], ref[ok]) < FP32_TOL
    assert_global_argmax(s, c, FP32_TOL)


def test_cdft_tile_spanning_more_lags_than_shared_buckets():
    """A 1000 km grid at 20 MHz: the one 64 x 64 node tile of each snapshot
    spans about 4900 lags, more than the 2048 shared-memory buckets of the
    histogram and the scatter, so both take their global-atomic path; the
    surface stays within the FP32 bound of the oracle."""
    s = sim.make_scene(seed=27, fs_hz=20e6, n_samples=20000, k_steps=2, fmt="ci16", waveform="noise",
                       snr_db=-3.0, grid_n=(41, 39), grid_spacing_m=25000.0, bw_hz=18e6)
    D, _ = oracle.node_geometry(s.grid, s.ephem, s.fs_hz, s.fc_hz)
    assert all(np.ptp(np.sign(d) * np.floor(np.abs(d) + 0.5)) >= 2048 for d in D)
    g, c = gpu_surface(s, algo="cdft")
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
    g.close()


@pytest.mark.parametrize("contract", ["fp32", "fp16x3"])
def test_cdft_superchunks(contract):
    """The combine sums chunks at the bin frequencies into super-chunks as
    long as the bin-spacing bound allows: a 4 km grid (narrow FDOA span)
    needs one super-chunk per snapshot; a 1000 km grid at 5 MHz with 64-sample
    chunks gets 4096-sample super-chunks (ten per snapshot). Both stay within
    the FP32 bound of the oracle."""
    for fs, spacing, chunk, one in ((12.5e6, 100.0, 256, True), (5e6, 25000.0, 64, False)):
        s = sim.make_scene(seed=25, fs_hz=fs, n_samples=40000, k_steps=2, fmt="ci16", waveform="chirp",
                           snr_db=-3.0, grid_n=(41, 39), grid_spacing_m=spacing)
        g, c = gpu_surface(s, algo="cdft", chunk=chunk, contract=contract)
        _, cand_chunks = g.cdft_work()
        if one:
            assert cand_chunks == s.G * s.k_steps
        else:
            assert s.G * s.k_steps < cand_chunks < s.G * s.k_steps * (40000 // chunk)
        ref = oracle_surface(s)
        ok = ~lag_boundary_mask(s, np.arange(s.G))
        assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
        g.close()


def test_cdft_rejects_chunk_too_long_for_the_bins():
    """A fixed chunk whose length times the bin spacing exceeds the
    interpolation bound (4096 samples on a 1000 km grid at 2 MHz: 0.085
    cycles) is refused with DG_EUNSUPPORTED when the surface is read; the
    context stays usable with a shorter chunk (1024: 0.021 cycles)."""
    torch = torch_cuda()
    P = package()
    s = sim.make_scene(seed=26, fs_hz=2e6, n_samples=20000, k_steps=1, fmt="ci16", waveform="chirp",
                       snr_db=-3.0, grid_n=(41, 39), grid_spacing_m=25000.0)
    g = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz, algo="cdft", chunk=4096)
    g.load_captures(s.fmt, torch.from_numpy(s.y1).cuda(), torch.from_numpy(s.y2).cuda())
    g.cost_surface()
    with pytest.raises(P.DGError) as e:
        g.sync()
    assert e.value.status == P.DG_EUNSUPPORTED
    g.close()
    g, c = gpu_surface(s, algo="cdft", chunk=1024)
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
    g.close()


@pytest.mark.parametrize("chunk", [64, 1024, 4096])
def test_cdft_chunk_sizes(chunk):
    s = sim.make_scene(seed=22, fs_hz=20e6, n_samples=9000, k_steps=2, fmt="ci8", waveform="noise",
                       snr_db=-3.0, grid_n=(33, 29), grid_spacing_m=400.0, bw_hz=18e6)
    g, c = gpu_surface(s, algo="cdft", chunk=chunk)
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
    g.close()


def test_cdft_mid_subgrid_full_k_n():
    s = sim.mid(grid_n=(49, 41))
    g, c = gpu_surface(s, algo="cdft")
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.ravel()[ok], ref.ravel()[ok]) < FP32_TOL
    assert_argmax_consistent(c, ref, FP32_TOL)
    g.close()


def _sampled(s, c, npts, seed, tol=FP32_TOL):
    """Pointwise bound on random nodes, then the complete argmax check over
    every node that can hold the oracle's maximum under that bound."""
    rng = np.random.default_rng(seed)
    idx = np.unique(rng.integers(0, s.G, npts))
    ref = oracle.cost_points(*oracle.scene_args(s), idx=idx)
    ok = ~lag_boundary_mask(s, idx)
    assert rel_err(c.ravel()[idx][ok], ref[ok]) < tol
    return assert_global_argmax(s, c, tol)


def test_cdft_mid_full_size_sampled_and_against_direct():
    s = sim.mid()
    g, c = gpu_surface(s, algo="cdft")
    _sampled(s, c, 48, 5)
    g.close()
    g, d = gpu_surface(s, algo="direct")
    assert rel_err(c, d) < 2 * FP32_TOL
    assert int(np.argmax(c.ravel())) == int(np.argmax(d.ravel()))
    g.close()


def test_cdft_large_full_size_sampled():
    s = sim.large()
    g, c = gpu_surface(s, algo="cdft")
    _sampled(s, c, 16, 6)
    g.close()


def test_cdft_refine_and_unsupported_options():
    torch = torch_cuda()
    P = package()
    s = sim.tiny(grid_n=41)
    g, _ = gpu_surface(s, algo="cdft")
    cost = g.cost_surface()
    fix = g.argmax_refine(cost, 100.0, 1000.0)
    ref = oracle_surface(s)
    # the 41 x 41 tiny surface's top two differ by ~1.9e-5 of the maximum: a
    # near-tie at the FP32 bound
    am = assert_argmax_consistent(cost.cpu().numpy(), ref, FP32_TOL, near_tie=True)
    lg = oracle.refine_grid(s.grid, fix["index"], 100.0, 1000.0)
    lref = oracle.cost_surface(lg, s.ephem, s.fs_hz, s.fc_hz, s.y1, s.y2)
    ri = fix["ri"] * lg["nlon"] + fix["rj"]
    assert lref.ravel()[ri] >= lref.max() * (1 - 2 * FP32_TOL)
    g.close()
    for kw in (dict(prec="fp64"), dict(chunk=100), dict(bins=32)):
        with pytest.raises(P.DGError):
            P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz, algo="cdft", **kw)


# --------------------------------------------------- tensor-core contraction
# Stated bounds of the 16-bit contractions against the FP64 oracle: the lag
# products and the DFT matrix are each rounded once to 16 bits (unit roundoff
# u = 2^-9 for bf16, 2^-11 for fp16) and the products are summed in FP32, so
# W carries a relative error of order 2u and |C|^2 about twice that:
# bf16 <= 1e-2, fp16 <= 2e-3 (about 2.5x the ~4u estimate). The split forms
# (16-bit high part + 16-bit residual, three products) leave ~3u^2 per
# product and are held to the FP32 bound itself.
TC_TOL = {"bf16": 1e-2, "fp16": 2e-3, "bf16x3": FP32_TOL, "fp16x3": FP32_TOL}


@pytest.mark.parametrize("contract", ["bf16", "fp16", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
def test_cdft_tensor_core_error_bounds(contract, fmt):
    s = sim.make_scene(seed=21, fs_hz=12.5e6, n_samples=3001, k_steps=3, fmt=fmt, waveform="chirp",
                       snr_db=-3.0, grid_n=(37, 45), grid_spacing_m=150.0)
    g, c = gpu_surface(s, algo="cdft", contract=contract)
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    err = rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01)
    assert err < TC_TOL[contract], err
    g.close()


@pytest.mark.parametrize("contract", ["bf16", "fp16", "bf16x3", "fp16x3"])
def test_cdft_tensor_core_mid_subgrid(contract):
    s = sim.mid(grid_n=(49, 41))
    g, c = gpu_surface(s, algo="cdft", contract=contract, chunk=1024)
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.ravel()[ok], ref.ravel()[ok]) < TC_TOL[contract]
    # the sub-grid's top two differ by ~1.1e-3 of the maximum: decisive at the
    # split forms' bound, a near-tie at the single 16-bit forms'
    assert_argmax_consistent(c, ref, TC_TOL[contract], near_tie=contract in ("bf16", "fp16"))
    g.close()


@pytest.mark.parametrize("contract", ["fp16", "fp16x3"])
def test_cdft_tensor_core_large_full_size_sampled(contract):
    s = sim.large()
    g, c = gpu_surface(s, algo="cdft", contract=contract, chunk=1024)
    rng = np.random.default_rng(7)
    idx = rng.integers(0, s.G, 16)
    ref = oracle.cost_points(*oracle.scene_args(s), idx=idx)
    ok = ~lag_boundary_mask(s, idx)
    assert rel_err(c.ravel()[idx][ok], ref[ok]) < TC_TOL[contract]
    g.close()


def test_tensor_pipeline_timeout_is_reported_and_the_context_recovers():
    """Every wait of the tensor-core pipeline is bounded. With the test hook
    lowering their poll limit to one poll, the first wait that is not already
    satisfied gives up: the kernel stops issuing, lets the MMAs and bulk
    copies it issued land, frees its tensor memory and returns, and the next
    synchronising call reports DG_ETIMEOUT. With the default limit restored,
    the same context's next surface matches the oracle."""
    torch = torch_cuda()
    P = package()
    s = sim.make_scene(seed=30, fs_hz=12.5e6, n_samples=8192, k_steps=2, fmt="ci16", waveform="chirp",
                       snr_db=-3.0, grid_n=(37, 45), grid_spacing_m=150.0)
    g = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz, algo="cdft", contract="fp16x3")
    g.load_captures(s.fmt, torch.from_numpy(s.y1).cuda(), torch.from_numpy(s.y2).cuda())
    try:
        P.dg_debug_tc_wait_limit(1)
        g.cost_surface()
        with pytest.raises(P.DGError) as e:
            g.sync()
        assert e.value.status == P.DG_ETIMEOUT
    finally:
        P.dg_debug_tc_wait_limit(0)
    c = g.cost_surface()
    g.sync()
    ref = oracle_surface(s)
    ok = ~lag_boundary_mask(s, np.arange(s.G))
    assert rel_err(c.double().cpu().numpy().ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
    g.close()


# ------------------------------------------------- fractional delay (Lagrange4)
@pytest.mark.parametrize("fmt", ["c64", "ci16", "ci8"])
@pytest.mark.parametrize("contract", ["fp32", "fp16x3"])
def test_cdft_lagrange4_small_scenes(fmt, contract):
    """The 4-tap Lagrange fractional delay (L = floor(D), mu = D - L) on the
    chunked-DFT path: by linearity each candidate combines the DFT rows of
    lags L - 1 .. L + 2 with its weights w_m(mu). Against the oracle's
    delay mode 1 (the definition, sample by sample) at the FP32 bound, with
    ragged tiles and odd N."""
    s = sim.make_scene(seed=31, fs_hz=12.5e6, n_samples=3001, k_steps=3, fmt=fmt, waveform="chirp",
                       snr_db=-3.0, grid_n=(37, 45), grid_spacing_m=150.0)
    g, c = gpu_surface(s, algo="cdft", contract=contract, delay="lagrange4")
    ref = oracle_surface(s, 1)
    ok = ~lag_boundary_mask(s, np.arange(s.G), 1)
    assert rel_err(c.ravel()[ok], ref.ravel()[ok], 0.01) < FP32_TOL
    g.close()


def test_cdft_lagrange4_mid_subgrid_and_noise_free_peak():
    """Mid geometry: on a 49 x 41 sub-grid at full K and N the Lagrange4
    surface matches the oracle (delay mode 1) within the FP32 bound and its
    maximum is a valid one (a near-tie); on the noise-free 21 x 21 scene the
    maximum is the emitter's node.""" 
    s = sim.mid(grid_n=(49, 41))
    g, c = gpu_surface(s, algo="cdft", delay="lagrange4")
    ref = oracle_surface(s, 1)
    ok = ~lag_boundary_mask(s, np.arange(s.G), 1)
    assert rel_err(c.ravel()[ok], ref.ravel()[ok]) < FP32_TOL
    # with the fractional delay the sub-grid's top two differ by ~5.8e-5 of
    # the maximum: a near-tie at the FP32 bound
    assert_argmax_consistent(c, ref, FP32_TOL, near_tie=True)
    g.close()
    s = sim.mid(grid_n=(21, 21), snr_db=None, waveform="noise", bw_hz=5e6)
    g, c = gpu_surface(s, algo="cdft", delay="lagrange4")
    ref = oracle_surface(s, 1)
    assert oracle.argmax(ref) == 10 * 21 + 10
    assert_argmax_consistent(c, ref, FP32_TOL)
    assert rel_err(c, ref) < FP32_TOL
    g.close()


def test_cdft_lagrange4_equals_direct_lagrange4_at_large_sizes():
    """Large footprint's captures on a 129 x 129 grid: the chunked-DFT
    Lagrange4 surface against the direct one (both FP32) and the oracle at
    sampled nodes."""
    s = sim.large(grid_n=129)
    g, c = gpu_surface(s, algo="cdft", delay="lagrange4")
    g.close()
    g, d = gpu_surface(s, algo="direct", delay="lagrange4")
    g.close()
    assert rel_err(c, d) < 2 * FP32_TOL
    rng = np.random.default_rng(8)
    idx = np.unique(rng.integers(0, s.G, 24))
    ref = oracle.cost_points(*oracle.scene_args(s), idx=idx, delay_mode=1)
    ok = ~lag_boundary_mask(s, idx, 1)
    assert rel_err(c.ravel()[idx][ok], ref[ok]) < FP32_TOL
