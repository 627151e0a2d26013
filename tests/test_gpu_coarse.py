"""Coarse delay-Doppler maps on the device (dg_coarse_maps) against the FP64
oracle (oracle/coarse.py): the per-snapshot parameters, every entry of the
map A, and the back-projected cell values.

Tolerances: the device sums M products per chunk and nb chunks per bin in
FP32, with twiddles accurate to about 1e-6 rad; for A = |X|^2 that is a
relative error of a few 1e-6 where |X| stands above the noise, and an error
of order 1e-7 mu at the noise floor (mu the map's mean). Both sides are held
to 1e-4 (A + mu). Cell values are maxima of the same entries over the same
boxes; a box is only compared where neither side could round it differently
(no corner lag within 1e-9 of a rounding boundary, no bin edge within 1e-9 of
an integer, by the FDOA tolerance below), since the two sides' geodetic
conversions may differ in the last bit and the device's FDOAs are FP32."""
import math

import numpy as np
import pytest

import oracle
import sim
from gpu_common import package, torch_cuda
from oracle import coarse as ocoarse

pytestmark = pytest.mark.gpu

# The device's node FDOAs come from double-float geometry (about 1e-11 cycles
# per sample) rounded to FP32 (6e-8 relative of |nu| < 1e-3): within 1e-10.
NU_TOL = 1e-10


def _scene(seed, grid_n, spacing, K, N, fmt, fs=5e6, waveform="noise", snr=0.0):
    return sim.make_scene(seed=seed, fs_hz=fs, n_samples=N, k_steps=K, fmt=fmt, waveform=waveform,
                          snr_db=snr, grid_n=grid_n, grid_spacing_m=spacing, bw_hz=0.8 * fs,
                          formation=sim.Formation(dt_s=5.0))


def _run(scene, bins=0, chunk=0):
    torch = torch_cuda()
    P = package()
    g = P.Geolocator(scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz)
    g.load_captures(scene.fmt, torch.from_numpy(scene.y1).cuda(), torch.from_numpy(scene.y2).cuda())
    maps = g.coarse_maps(bins=bins, chunk=chunk)
    A, steps, (Q, M, cap) = g.coarse_inspect()
    out = maps.double().cpu().numpy(), A.double().cpu().numpy(), steps, (Q, M, cap)
    g.close()
    return out


def _unambiguous(scene, Q):
    """Cells whose delay-Doppler box both sides must compute the same way."""
    D, nu = oracle.node_geometry(scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz)
    fr = np.abs(D) - np.floor(np.abs(D))
    near_lag = np.abs(fr - 0.5) < 1e-9
    ok = []
    for k in range(D.shape[0]):
        lag = ocoarse.round_half_away(D[k])
        l0, nlag, lo, delta, nc = ocoarse.step_params(lag, nu[k], Q)
        nl = near_lag[k]
        bad_lag = nl[:-1, :-1] | nl[1:, :-1] | nl[:-1, 1:] | nl[1:, 1:]
        v = np.stack([nu[k][:-1, :-1], nu[k][1:, :-1], nu[k][:-1, 1:], nu[k][1:, 1:]])
        xs = [(v.min(axis=0) - lo) / delta, (v.max(axis=0) - lo) / delta] if delta > 0 else []
        bad_bin = np.zeros_like(bad_lag)
        tau = 4 * NU_TOL / delta if delta > 0 else 0.0
        for x in xs:
            # the extreme bins (x = 0 at nu_lo, x = Q - 1 at nu_hi after the
            # clip) come out the same on both sides by construction
            bad_bin |= (np.abs(x - np.rint(x)) < tau) & (x > tau) & (x < Q - 1 - tau)
        ok.append(~(bad_lag | bad_bin))
    return np.stack(ok)


CASES = [
    # seed, nodes (lat, lon), spacing m, K, N, format, bins, chunk
    (21, (21, 25), 2000.0, 3, 5000, "c64", 0, 0),        # auto bins / chunk, N not a multiple of M
    (22, (9, 7), 5000.0, 2, 3000, "ci16", 24, 64),       # ragged everything, int16
    (23, (41, 41), 25000.0, 2, 4096, "ci8", 16, 256),   # > 896 lags at 20 MHz: several lag tiles
    (24, (5, 6), 3000.0, 2, 700, "c64", 9, 1),           # chunk 1: the exact Eq. 11 CAF
]


@pytest.mark.parametrize("case", CASES, ids=[f"seed{c[0]}" for c in CASES])
def test_coarse_maps_match_the_oracle(case):
    seed, nodes, spacing, K, N, fmt, bins, chunk = case
    s = _scene(seed, nodes, spacing, K, N, fmt, fs=20e6 if seed == 23 else 5e6)
    maps, A, steps, (Q, M, cap) = _run(s, bins, chunk)
    if bins:
        assert Q == bins
    if chunk:
        assert M == chunk
    ref_maps, extra = ocoarse.coarse_maps(s.grid, s.ephem, s.fs_hz, s.fc_hz, s.y1, s.y2, Q, M, want_caf=True)
    for k in range(K):
        (l0, nlag, lo, delta, nc), RA, mu = extra[k]
        st = steps[k]
        assert (st["l0"], st["nlag"]) == (l0, nlag)
        # node FDOAs: double-float geometry rounded to FP32 on the device
        assert abs(st["nu_lo"] - lo) <= NU_TOL
        assert abs(st["delta"] - delta) <= 2 * NU_TOL / (Q - 1)
        assert abs(st["nu_c"] - nc) <= NU_TOL
        assert st["mu"] == pytest.approx(mu, rel=1e-5)
        assert nlag <= cap
        err = np.abs(A[k, :nlag] - RA) / (RA + mu)
        assert err.max() <= 1e-4, f"snapshot {k}: max A error {err.max():.2e}"
    ok = _unambiguous(s, Q)
    assert ok.mean() > 0.95
    err = np.abs(maps - ref_maps) / (ref_maps + 1.0)
    assert err[ok].max() <= 1e-4, f"max cell error {err[ok].max():.2e}"
    if seed == 23:
        assert extra[0][0][1] > 896


def test_coarse_peak_sits_on_the_emitter():
    """Noise-free wideband emitter on the centre node: in every snapshot the
    four cells around it reach the map's largest value."""
    s = _scene(25, (31, 31), 1000.0, 3, 4096, "c64", snr=None)
    maps, _, _, _ = _run(s)
    for k in range(3):
        top = maps[k].max()
        assert maps[k, 14:16, 14:16].max() == pytest.approx(top, rel=1e-6)


def test_coarse_errors():
    torch = torch_cuda()
    P = package()
    s = _scene(26, (9, 9), 2000.0, 2, 1024, "c64")
    g = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz)
    with pytest.raises(P.DGError, match="status 4"):
        g.coarse_inspect()
    with pytest.raises(P.DGError, match="status 4"):
        g.coarse_maps()  # captures not loaded
    g.load_captures(s.fmt, torch.from_numpy(s.y1).cuda(), torch.from_numpy(s.y2).cuda())
    with pytest.raises(P.DGError, match="status 1"):
        g.coarse_maps(bins=1)
    with pytest.raises(P.DGError, match="status 1"):
        g.coarse_maps(chunk=48)
    g.coarse_maps()
    g.sync()
    g.close()
    shard = P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz, row0=2, nrows=4)
    shard.load_captures(s.fmt, torch.from_numpy(s.y1).cuda(), torch.from_numpy(s.y2).cuda())
    with pytest.raises(P.DGError, match="status 6"):
        shard.coarse_maps(out=torch.empty((2, 8, 8), device="cuda"))
    shard.close()
