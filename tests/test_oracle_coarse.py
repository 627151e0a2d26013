"""Pins of the coarse-map oracle (oracle/coarse.py) to things other than
itself: the Eq. 11 correlation of the C oracle, exactness where the chunked
form is exact, its error bound elsewhere, a noise-free peak at the true delay
and Doppler, and the max-pool bound checked against a fine lattice of points
inside every cell."""
import math

import numpy as np
import pytest

import oracle
import sim
from oracle import coarse


def _pair(seed, N, l0=7, nu0=2.5e-3, snr=None):
    """y2[n + l0] = y1[n] exp(j 2 pi nu0 n) (plus noise), receiver 2 shifted
    by the FDOA nu0 relative to receiver 1 (Eq. 1): the correlation
    y1[n] conj(y2[n + l0]) exp(j 2 pi nu0 n) is |y1[n]|^2, in phase."""
    rng = np.random.default_rng(seed)
    y1 = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) / math.sqrt(2)
    y2 = np.zeros(N, dtype=np.complex128)
    n = np.arange(N)
    y2[l0:] = (y1 * np.exp(2j * math.pi * nu0 * n))[:N - l0]
    if snr is not None:
        y2 += (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * math.sqrt(0.5 / snr)
    return y1, y2


def test_m1_equals_the_eq11_correlation():
    """M = 1: every entry is |C|^2 of the C oracle's Eq. 11 at that lag and
    bin frequency."""
    y1, y2 = _pair(1, 300, snr=0.5)
    l0, nlag, lo, Q = -4, 15, -3e-3, 9
    delta = 0.9e-3
    A = coarse.caf(y1, y2, l0, nlag, lo, delta, lo + 0.37e-3, Q, 1)
    for t in range(nlag):
        for q in range(Q):
            c = oracle.correlate(y1, y2, float(l0 + t), lo + q * delta)
            assert A[t, q] == pytest.approx(abs(c) ** 2, rel=1e-11, abs=1e-9)


@pytest.mark.parametrize("M", [4, 16, 64])
def test_chunked_form_exact_at_the_centre_and_bounded_elsewhere(M):
    y1, y2 = _pair(2, 1000, snr=1.0)
    l0, nlag, lo, hi, Q = 3, 9, 1.0e-3, 4.0e-3, 7
    delta, nc = (hi - lo) / (Q - 1), 0.5 * (lo + hi)
    A = coarse.caf(y1, y2, l0, nlag, lo, delta, nc, Q, M)
    for t in range(nlag):
        l = l0 + t
        y2s = np.zeros_like(y2)
        y2s[:1000 - l] = y2[l:]
        s_abs = np.sum(np.abs(y1) * np.abs(y2s))
        for q in range(Q):
            nu_q = lo + q * delta
            c = oracle.correlate(y1, y2, float(l), nu_q)
            if q == (Q - 1) // 2:  # nu_q = nu_c up to rounding
                assert A[t, q] == pytest.approx(abs(c) ** 2, rel=1e-9, abs=1e-9)
            bound = 2 * math.pi * abs(nu_q - nc) * (M - 1) * s_abs
            assert abs(math.sqrt(A[t, q]) - abs(c)) <= bound * (1 + 1e-9) + 1e-9
    # the bound is not vacuous: far bins do move
    c_edge = oracle.correlate(y1, y2, float(l0 + 4), lo)
    assert abs(math.sqrt(A[4, 0]) - abs(c_edge)) > 0.0 or M == 1


def test_noise_free_peak_at_the_true_delay_and_doppler():
    """Noise-free shifted copy: the map's maximum is at (l0, nu0), where it
    reaches the Cauchy-Schwarz value (sum of |y1|^2 over the overlap)^2."""
    N, l0, nu0 = 2048, 9, 1.5e-3
    y1, y2 = _pair(3, N, l0, nu0)
    Q = 13
    lo, hi = nu0 - 6 * 2.5e-4, nu0 + 6 * 2.5e-4  # nu0 is the centre bin
    A = coarse.caf(y1, y2, 0, 20, lo, (hi - lo) / (Q - 1), 0.5 * (lo + hi), Q, 32)
    t, q = np.unravel_index(np.argmax(A), A.shape)
    assert (t, q) == (l0, 6)
    cs = np.sum(np.abs(y1[:N - l0]) ** 2) ** 2
    assert A[l0, 6] == pytest.approx(cs, rel=1e-12)


def test_backprojection_bounds_every_point_inside_the_cell():
    """For points on a 5 x 5 lattice inside each cell (the fine grid at a
    quarter of the spacing), the lag round(D) and the FDOA lie inside the
    cell's box, and A at that lag and both bins around the FDOA is at most
    the cell's coarse value times mu."""
    s = sim.tiny(seed=11, n_samples=2048, snr_db=0.0)
    grid = dict(s.grid, nlat=9, nlon=9, dlat_m=4000.0, dlon_m=4000.0)
    fine = dict(grid, nlat=33, nlon=33, dlat_m=1000.0, dlon_m=1000.0)
    Q, M = 16, 64
    maps, extra = coarse.coarse_maps(grid, s.ephem, s.fs_hz, s.fc_hz, s.y1, s.y2, Q, M, want_caf=True)
    (l0, nlag, lo, delta, nc), A, mu = extra[0]
    Df, nuf = oracle.node_geometry(fine, s.ephem, s.fs_hz, s.fc_hz)
    Lf = coarse.round_half_away(Df[0])
    checked = 0
    for i in range(8):
        for j in range(8):
            v = maps[0, i, j] * mu
            for a in range(5):
                for b in range(5):
                    L, nu = int(Lf[4 * i + a, 4 * j + b]), nuf[0, 4 * i + a, 4 * j + b]
                    assert 0 <= L - l0 < nlag
                    x = (nu - lo) / delta
                    for q in (math.floor(x), math.ceil(x)):
                        q = min(max(q, 0), Q - 1)
                        assert A[L - l0, q] <= v * (1 + 1e-12)
                        checked += 1
    assert checked == 8 * 8 * 25 * 2


def test_backprojection_constant_and_zero_maps():
    lag = np.array([[3, 4], [4, 6]])
    nu = np.array([[1e-3, 2e-3], [1.5e-3, 2.5e-3]])
    A = np.full((4, 5), 2.5)
    assert coarse.backproject(A, 2.5, lag, nu, 3, 1e-3, 3.75e-4)[0, 0] == 1.0
    assert coarse.backproject(np.zeros((4, 5)), 0.0, lag, nu, 3, 1e-3, 3.75e-4)[0, 0] == 0.0
    # a spike outside the cell's box does not show; inside it does
    A = np.ones((4, 5))
    A[0, 0] = 50.0
    mu = A.mean()
    assert coarse.backproject(A, mu, lag, nu, 3, 1e-3, 3.75e-4)[0, 0] == pytest.approx(50.0 / mu)
    A = np.ones((4, 5))
    A[2, 0] = 50.0  # lag 5 is inside [3, 6], bin 0 is inside [0, 4]
    assert coarse.backproject(A, A.mean(), lag, nu, 3, 1e-3, 3.75e-4)[0, 0] == pytest.approx(50.0 / A.mean())
    A = np.ones((8, 5))
    A[7, 2] = 50.0  # lag 10 is outside [3, 6]
    assert coarse.backproject(A, A.mean(), lag, nu, 3, 1e-3, 3.75e-4)[0, 0] == pytest.approx(1.0 / A.mean())


def test_round_half_away_from_zero():
    D = np.array([-2.5, -1.5, -0.5, -0.49999999999999994, 0.0, 0.49999999999999994, 0.5, 1.5, 2.5, 2.4999999])
    assert coarse.round_half_away(D).tolist() == [-3, -2, -1, 0, 0, 0, 1, 2, 3, 2]
