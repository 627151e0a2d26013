"""Pins of the CPU oracle to things other than itself.

Each pin is a plain function that raises AssertionError when the oracle
disagrees with a closed form, a published constant, a numpy/FFT library
routine or an exact invariant. ``test_oracle_pins.py`` runs every pin against
the oracle; ``test_oracle_mutants.py`` runs them against copies of the oracle
source with one planted mistake each and requires that some pin fails.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle
import sim

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RNG_SEED = 1234


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _rand_iq(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# ----------------------------------------------------------------- geodesy
def pin_wgs84_published_constants():
    """Pole, equator and height map to the published WGS-84 axes."""
    g = _golden("wgs84.json")
    pole = oracle.geodetic_to_ecef(math.pi / 2, 0.0)
    assert abs(pole[2] - g["b_m"]) < g["b_tolerance_m"], pole
    assert abs(pole[0]) < 1e-6 and abs(pole[1]) < 1e-6, pole
    eq = oracle.geodetic_to_ecef(0.0, 0.0)
    assert np.allclose(eq, [g["a_m"], 0.0, 0.0], rtol=0, atol=1e-9), eq
    eq90 = oracle.geodetic_to_ecef(0.0, math.pi / 2)
    assert np.allclose(eq90, [0.0, g["a_m"], 0.0], rtol=0, atol=1e-9), eq90
    up = oracle.geodetic_to_ecef(0.0, 0.0, 1000.0)
    assert abs(up[0] - g["a_m"] - 1000.0) < 1e-9, up
    e2 = 1.0 - (g["b_m"] / g["a_m"]) ** 2
    assert abs(e2 - g["e2"]) < 1e-10  # fixture self-consistency (b is printed to 0.1 mm)


def pin_ellipsoid_invariants():
    """h = 0 points lie on the ellipsoid; the surface normal there has the
    geodetic latitude as elevation and the longitude as azimuth; height moves
    along that normal."""
    g = _golden("wgs84.json")
    a, b = g["a_m"], g["b_m"]
    rng = np.random.default_rng(RNG_SEED)
    for lat, lon in zip(rng.uniform(-89.0, 89.0, 16), rng.uniform(-179.0, 179.0, 16)):
        la, lo = math.radians(lat), math.radians(lon)
        p = oracle.geodetic_to_ecef(la, lo)
        x, y, z = p
        assert abs((x * x + y * y) / (a * a) + z * z / (b * b) - 1.0) < 1e-10
        nx, ny, nz = x / a ** 2, y / a ** 2, z / b ** 2
        assert abs(math.atan2(nz, math.hypot(nx, ny)) - la) < 1e-9
        assert abs(math.atan2(y, x) - lo) < 1e-12
        ph = oracle.geodetic_to_ecef(la, lo, 2500.0)
        n_hat = np.array([math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)])
        assert np.allclose(ph - p, 2500.0 * n_hat, rtol=0, atol=1e-7)


def pin_grid_nodes():
    """Centre node is (lat0, lon0); nodes are evenly spaced; spacing is metres
    on the ellipsoid (meridian arc, parallel arc) at the centre latitude;
    grid_ecef is the per-node conversion."""
    grid = dict(lat0_deg=40.0, lon0_deg=-100.0, dlat_m=1000.0, dlon_m=700.0, nlat=5, nlon=7)
    la, lo = oracle.grid_node(grid, 2, 3)
    assert la == math.radians(40.0) and lo == math.radians(-100.0)
    lam, _ = oracle.grid_node(grid, 1, 3)
    lap, _ = oracle.grid_node(grid, 3, 3)
    assert abs((lap - la) - (la - lam)) < 1e-15
    p = {ij: oracle.geodetic_to_ecef(*oracle.grid_node(grid, *ij)) for ij in [(1, 3), (3, 3), (2, 2), (2, 4)]}
    d_lat = np.linalg.norm(p[(3, 3)] - p[(1, 3)])
    d_lon = np.linalg.norm(p[(2, 4)] - p[(2, 2)])
    assert abs(d_lat / 2000.0 - 1.0) < 1e-7, d_lat
    assert abs(d_lon / 1400.0 - 1.0) < 1e-7, d_lon
    xyz = oracle.grid_ecef(grid)
    assert xyz.shape == (35, 3)
    for i, j in [(0, 0), (4, 6), (2, 5)]:
        assert np.array_equal(xyz[i * 7 + j], oracle.geodetic_to_ecef(*oracle.grid_node(grid, i, j)))
    # the paper's sizing example (Sec. I): 10 x 10 deg at 0.01 deg ~ a million values
    pp = _golden("paper_parameters.json")
    n_side = int(round(pp["grid_extent_deg"] / pp["grid_spacing_deg"])) + 1
    assert abs(n_side * n_side / pp["grid_values_approx"] - 1.0) < 0.01


# ---------------------------------------------------------------- geometry
def _circular_case(phi1, phi2, psi, beta, a=6.928e6, R=6.371e6, gm=3.986004418e14):
    n = math.sqrt(gm / a ** 3)
    eph = np.array([a * math.cos(phi1), a * math.sin(phi1), 0.0,
                    -n * a * math.sin(phi1), n * a * math.cos(phi1), 0.0,
                    a * math.cos(phi2), a * math.sin(phi2), 0.0,
                    -n * a * math.sin(phi2), n * a * math.cos(phi2), 0.0])
    pe = R * np.array([math.cos(beta) * math.cos(psi), math.cos(beta) * math.sin(psi), math.sin(beta)])
    rho = [math.sqrt(a * a + R * R - 2 * a * R * math.cos(beta) * math.cos(ph - psi)) for ph in (phi1, phi2)]
    rdot = [a * R * n * math.cos(beta) * math.sin(ph - psi) / r for ph, r in zip((phi1, phi2), rho)]
    return eph, pe, rho, rdot


def pin_geometry_circular_orbit():
    """Eq. 3-8 against the closed form for receivers on a circular orbit in
    the x-y plane around a non-rotating sphere."""
    fs, fc = 12.5e6, 1575.42e6
    lam = sim.C_LIGHT / fc
    rng = np.random.default_rng(RNG_SEED)
    for _ in range(12):
        phi1 = rng.uniform(0, 2 * math.pi)
        phi2 = phi1 + rng.uniform(0.002, 0.02)
        psi = phi1 + rng.uniform(-0.1, 0.1)
        beta = rng.uniform(-0.1, 0.1)
        eph, pe, rho, rdot = _circular_case(phi1, phi2, psi, beta)
        dtau, dfreq, D, nu = oracle.geometry(pe, eph, fs, fc)
        f = [-r / lam for r in rdot]
        want_dtau = (rho[1] - rho[0]) / sim.C_LIGHT
        assert abs(dtau - want_dtau) < 1e-9 * abs(rho[0] / sim.C_LIGHT), (dtau, want_dtau)
        assert abs(dfreq - (f[1] - f[0])) < 1e-6 * max(1.0, abs(f[0])), (dfreq, f)
        assert abs(D - want_dtau * fs) < 1e-6, D
        assert abs(nu - (f[1] - f[0]) / fs) < 1e-12


def pin_geometry_midpoint_special_case():
    """Emitter on the bisector of the two receivers: zero TDOA (lag 0) and
    opposite Dopplers, so the FDOA is twice receiver 2's Doppler."""
    fs, fc = 5e6, 1575.42e6
    lam = sim.C_LIGHT / fc
    phi1, phi2 = 0.4, 0.4072
    eph, pe, rho, rdot = _circular_case(phi1, phi2, 0.5 * (phi1 + phi2), 0.05)
    dtau, dfreq, D, nu = oracle.geometry(pe, eph, fs, fc)
    assert abs(D) < 1e-6 and int(np.round(D)) == 0
    f2 = -rdot[1] / lam
    assert abs(rdot[0] + rdot[1]) < 1e-9 * abs(rdot[0])
    assert abs(dfreq - 2 * f2) < 1e-6, (dfreq, f2)


def pin_geometry_matches_orbit_finite_difference():
    """Against the simulator's independent truth: delay from range / c,
    Doppler from a finite-difference range rate along the propagated orbit."""
    form = sim.Formation()
    fc, fs = 1575.42e6, 5e6
    rng = np.random.default_rng(RNG_SEED)
    for k in range(3):
        t = 3.0 * k
        lat, lon = sim.pick_emitter(rng, form, t)
        pe = sim.geodetic_to_ecef(lat, lon)
        eph = np.concatenate(form.states(t))
        tau, fd = sim.truth_delay_doppler(form, t, pe, fc)
        dtau, dfreq, D, nu = oracle.geometry(pe, eph, fs, fc)
        assert abs(dtau - (tau[1] - tau[0])) < 1e-15, (dtau, tau)
        assert abs(dfreq - (fd[1] - fd[0])) < 1e-4, (dfreq, fd)


# ------------------------------------------------------------- correlation
def pin_lagrange_reproduces_cubics():
    """The 4-tap weights at taps -1..2 interpolate every cubic exactly."""
    taps = np.array([-1.0, 0.0, 1.0, 2.0])
    for mu in np.linspace(0.0, 0.999, 11):
        w = oracle.lagrange4(mu)
        for p in range(4):
            assert abs(np.dot(w, taps ** p) - mu ** p) < 1e-13, (mu, p, w)
    assert np.array_equal(oracle.lagrange4(0.0), [0.0, 1.0, 0.0, 0.0])


def pin_correlate_vdot():
    """Zero lag, zero FDOA: Eq. 11 is numpy's conjugating inner product."""
    rng = np.random.default_rng(RNG_SEED)
    y1, y2 = _rand_iq(rng, 257), _rand_iq(rng, 257)
    c = oracle.correlate(y1, y2, 0.0, 0.0)
    want = np.vdot(y2, y1)
    assert abs(c - want) < 1e-12 * abs(want) * 10, (c, want)


def pin_correlate_lags_numpy_correlate():
    """Zero FDOA: the integer-lag sum equals numpy.correlate's full output at
    the lag given by Eq. 9 (round half away from zero)."""
    rng = np.random.default_rng(RNG_SEED)
    n = 200
    y1, y2 = _rand_iq(rng, n), _rand_iq(rng, n)
    full = np.correlate(y1, y2, "full")  # full[k + n - 1] = sum_m y1[m + k] conj(y2[m])
    for D, L in [(0.2, 0), (-0.49, 0), (3.0, 3), (2.5, 3), (-2.5, -3), (-17.4, -17), (199.0, 199), (-199.0, -199)]:
        c = oracle.correlate(y1, y2, D, 0.0)
        want = full[n - 1 - L]
        assert abs(c - want) <= 1e-12 * (abs(want) + 1.0) * 10, (D, L, c, want)
    assert abs(oracle.correlate(y1, y2, 250.0, 0.0)) == 0.0


def pin_correlate_fft_bins():
    """FDOA on DFT bins m / N: Eq. 11 equals N * ifft of the lag product."""
    rng = np.random.default_rng(RNG_SEED)
    n = 256
    y1, y2 = _rand_iq(rng, n), _rand_iq(rng, n)
    for L in (0, 5, -9):
        z = np.zeros(n, dtype=complex)
        lo, hi = max(0, -L), min(n, n - L)
        z[lo:hi] = y1[lo:hi] * np.conj(y2[lo + L:hi + L])
        spec = n * np.fft.ifft(z)
        for m in (0, 1, 7, -3, 100):
            c = oracle.correlate(y1, y2, float(L), m / n)
            assert abs(c - spec[m % n]) < 1e-9 * (abs(spec[m % n]) + 1.0), (L, m, c, spec[m % n])


def pin_correlate_tone_closed_form():
    """Two tones: a geometric series, C = exp(-j2pi fb L/fs) *
    exp(j pi d (2 n0 + M - 1)) sin(pi M d) / sin(pi d) over the M = N - |L|
    overlapping samples starting at n0, with d = (fa - fb)/fs + nu."""
    fs, n = 5e6, 1000
    t = np.arange(n) / fs
    for fa, fb, L, nu in [(1e3, -2e3, 7, 1.3e-4), (0.0, 5e3, -12, -4e-4), (2.5e4, 2.5e4, 0, 3e-5)]:
        y1, y2 = np.exp(2j * np.pi * fa * t), np.exp(2j * np.pi * fb * t)
        c = oracle.correlate(y1, y2, float(L), nu)
        d = (fa - fb) / fs + nu
        m = n - abs(L)
        n0 = max(0, -L)
        want = (np.exp(-2j * np.pi * fb * L / fs) * np.exp(1j * np.pi * d * (2 * n0 + m - 1))
                * math.sin(math.pi * m * d) / math.sin(math.pi * d))
        assert abs(c - want) < 1e-9 * m, (fa, fb, L, nu, c, want)


def pin_lagrange_mode_linearity():
    """Fractional mode is the weighted sum of integer-mode correlations at the
    four taps (interpolation is linear with real weights); at mu = 0 it equals
    the integer mode."""
    rng = np.random.default_rng(RNG_SEED)
    n = 300
    y1, y2 = _rand_iq(rng, n), _rand_iq(rng, n)
    for D, nu in [(4.3, 2e-3), (-6.75, -1e-3), (0.5, 0.0), (297.2, 1e-4)]:
        L = math.floor(D)
        w = oracle.lagrange4(D - L)
        want = sum(w[m + 1] * oracle.correlate(y1, y2, float(L + m), nu) for m in range(-1, 3))
        c = oracle.correlate(y1, y2, D, nu, delay_mode=1)
        assert abs(c - want) < 1e-10 * (abs(want) + 1.0), (D, c, want)
    assert oracle.correlate(y1, y2, 3.0, 1e-3, 1) == oracle.correlate(y1, y2, 3.0, 1e-3, 0)


# ------------------------------------------------------- surface and argmax
def _tiny_noise_scene(**kw):
    args = dict(seed=11, fs_hz=5e6, n_samples=1024, k_steps=2, fmt="c64", waveform="noise",
                snr_db=None, grid_n=9, grid_spacing_m=1500.0, bw_hz=2e6, integer_delays=True)
    args.update(kw)
    return sim.make_scene(**args)


def pin_swap_receivers():
    """Exchanging the receivers negates lag and FDOA and conjugates C up to a
    phase, so |C| and the whole surface are unchanged (integer mode)."""
    s = _tiny_noise_scene(snr_db=0.0, integer_delays=False)
    eph2 = np.concatenate([s.ephem[:, 6:], s.ephem[:, :6]], axis=1)
    a = oracle.cost_surface(s.grid, s.ephem, s.fs_hz, s.fc_hz, s.y1, s.y2)
    b = oracle.cost_surface(s.grid, eph2, s.fs_hz, s.fc_hz, s.y2, s.y1)
    assert np.allclose(a, b, rtol=1e-9, atol=0), np.max(np.abs(a - b) / a)


def pin_noise_free_peak():
    """Noise-free captures with whole-sample delays: the emitter's cell is the
    argmax and reaches the Cauchy-Schwarz bound of its overlap (the matched
    correlation of Sec. III)."""
    s = _tiny_noise_scene(k_steps=1, grid_n=11)
    cost = oracle.cost_surface(*oracle.scene_args(s))
    centre = (s.grid["nlat"] // 2) * s.grid["nlon"] + s.grid["nlon"] // 2
    assert oracle.argmax(cost) == centre
    y1, y2 = s.y_complex(1)[0], s.y_complex(2)[0]
    L = int(np.rint((s.tau[0, 1] - s.tau[0, 0]) * s.fs_hz))
    n = s.n_samples
    lo, hi = max(0, -L), min(n, n - L)
    bound = np.sum(np.abs(y1[lo:hi]) ** 2) * np.sum(np.abs(y2[lo + L:hi + L]) ** 2)
    assert abs(cost.ravel()[centre] / bound - 1.0) < 1e-9, cost.ravel()[centre] / bound


def pin_accumulation_and_modes():
    """Algorithm 1 sums the per-snapshot grids: the K = 2 surface is the sum
    of the two single-snapshot surfaces; magnitude mode sums |C_k|."""
    s = _tiny_noise_scene(snr_db=-3.0, integer_delays=False, grid_n=5)
    args = (s.grid, s.ephem, s.fs_hz, s.fc_hz)
    both = oracle.cost_surface(*args, s.y1, s.y2)
    one = [oracle.cost_surface(s.grid, s.ephem[k:k + 1], s.fs_hz, s.fc_hz, s.y1[k:k + 1], s.y2[k:k + 1])
           for k in range(2)]
    assert np.array_equal(both, one[0] + one[1])
    mag = oracle.cost_surface(*args, s.y1, s.y2, acc_mode=1)
    magk = [oracle.cost_surface(s.grid, s.ephem[k:k + 1], s.fs_hz, s.fc_hz, s.y1[k:k + 1], s.y2[k:k + 1],
                                acc_mode=1) for k in range(2)]
    assert np.allclose(magk[0], np.sqrt(one[0]), rtol=1e-15, atol=0)
    assert np.allclose(mag, magk[0] + magk[1], rtol=1e-15, atol=0)


def pin_argmax_ties_and_nan():
    assert oracle.argmax(np.array([1.0, 3.0, 3.0, 2.0])) == 1
    assert oracle.argmax(np.array([np.nan, 1.0, np.nan, 0.5])) == 1
    assert oracle.argmax(np.array([np.nan, np.nan])) == -1
    assert oracle.argmax(np.array([-5.0, -5.0])) == 0


def _bumps(shape, centres, amps, width=1.5):
    ii, jj = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    v = np.zeros(shape)
    for (ci, cj), a in zip(centres, amps):
        v += a * np.exp(-((ii - ci) ** 2 + (jj - cj) ** 2) / (2 * width * width))
    return v


def pin_detect_known_bumps():
    """Algorithm 1's threshold step on a surface of separated Gaussian bumps:
    exactly the bump centres pass, strongest first; the threshold and
    max_peaks cut from the weak end; a value equal to the threshold passes."""
    centres, amps = [(5, 40), (30, 7), (33, 44), (0, 0)], [5.0, 3.0, 1.0, 2.0]
    v = _bumps((41, 53), centres, amps)
    order = [centres[k][0] * 53 + centres[k][1] for k in np.argsort(amps)[::-1]]
    assert list(oracle.detect(v, 0.5, 3)) == order
    assert list(oracle.detect(v, 2.5, 3)) == order[:2]
    assert list(oracle.detect(v, 0.5, 3, max_peaks=1)) == order[:1]
    assert list(oracle.detect(v, float(v[0, 0]), 3)) == order[:3]
    assert list(oracle.detect(v, np.nextafter(v[0, 0], np.inf), 3)) == order[:2]


def pin_detect_plateau_edges_radius():
    """A flat top gives one peak, at its lowest linear index; windows clip at
    the grid edge; radius 0 makes every node above the threshold a peak;
    a wider window suppresses a lower neighbour bump."""
    v = np.zeros((9, 11))
    v[3:6, 4:7] = 2.0
    v[8, 10] = 1.0
    assert list(oracle.detect(v, 0.5, 2)) == [3 * 11 + 4, 8 * 11 + 10]
    assert len(oracle.detect(v, 0.5, 0)) == 10
    w = _bumps((21, 21), [(10, 5), (10, 9)], [2.0, 1.0], width=0.8)
    assert list(oracle.detect(w, 0.1, 2)) == [10 * 21 + 5, 10 * 21 + 9]
    assert list(oracle.detect(w, 0.1, 4)) == [10 * 21 + 5]


def pin_detect_matches_maximum_filter():
    """On continuous random surfaces (no ties), a peak is exactly a node
    equal to scipy's maximum filter over the (2r+1)^2 window (edges padded
    with -inf) and at least the threshold."""
    from scipy import ndimage
    rng = np.random.default_rng(11)
    for shape, r in (((17, 23), 1), ((30, 12), 2), ((25, 25), 3)):
        v = ndimage.gaussian_filter(rng.standard_normal(shape), 1.0)
        thr = float(np.quantile(v, 0.6))
        mf = ndimage.maximum_filter(v, size=2 * r + 1, mode="constant", cval=-np.inf)
        want = np.flatnonzero((v == mf) & (v >= thr))
        want = want[np.lexsort((want, -v.ravel()[want]))]
        assert list(oracle.detect(v, thr, r, max_peaks=1000)) == list(want)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_") and callable(v)]
