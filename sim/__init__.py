"""Seeded synthetic captures for direct geolocation (input generator only).

This module is the forward model that produces inputs for both the CPU oracle
and the CUDA library. It holds none of the estimator's arithmetic: no
per-candidate TDOA/FDOA, no correlation, no accumulation, no argmax.

What it models (Sec. II, Eq. 1-2; Sec. IV-A waveforms, Eq. 12):

* two LEO receivers on one circular orbit, receiver 2 leading receiver 1 by a
  fixed along-track arc, propagated in an inertial frame and rotated into ECEF;
* one stationary emitter on the WGS-84 ellipsoid;
* a baseband waveform x(t) (band-limited complex Gaussian noise, a chirp, a
  sawtooth or a pure tone at the carrier);
* what receiver i records, per Eq. 1 with delay and Doppler held constant over
  a snapshot: y_i[n] = A x(n T_s - tau_i) exp(j 2 pi f_i n T_s) + w_i[n].

The true delay is geometric range / c. The true Doppler is minus the range
rate over the wavelength, where the range rate comes from a central finite
difference of the range along the propagated orbit (not from a closed form),
so this module is an independent check on the geometry used elsewhere.

Everything is seeded (numpy PCG64); nothing is read from disk.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0
WGS84_A = 6_378_137.0
WGS84_F = 1.0 / 298.257223563
WGS84_E2 = WGS84_F * (2.0 - WGS84_F)
OMEGA_E = 7.2921150e-5
GM_EARTH = 3.986004418e14

FORMATS = ("c64", "ci16", "ci8")
FORMAT_CODE = {"c64": 0, "ci16": 1, "ci8": 2}


# --------------------------------------------------------------------------
# geodesy and orbits (forward model)
# --------------------------------------------------------------------------
def geodetic_to_ecef(lat_deg, lon_deg, h=0.0):
    """WGS-84 geodetic (deg, deg, m) -> ECEF metres, numpy-vectorised."""
    lat = np.radians(np.asarray(lat_deg, dtype=np.float64))
    lon = np.radians(np.asarray(lon_deg, dtype=np.float64))
    s = np.sin(lat)
    n_pv = WGS84_A / np.sqrt(1.0 - WGS84_E2 * s * s)
    x = (n_pv + h) * np.cos(lat) * np.cos(lon)
    y = (n_pv + h) * np.cos(lat) * np.sin(lon)
    z = (n_pv * (1.0 - WGS84_E2) + h) * s
    return np.stack([x, y, z], axis=-1)


def orbit_state_ecef(t, radius, incl, raan, u0):
    """Circular Keplerian orbit: ECEF position and velocity at time t (s).

    The inertial and Earth-fixed frames coincide at t = 0; the Earth-fixed
    frame then turns at OMEGA_E about +z.
    """
    n = math.sqrt(GM_EARTH / radius ** 3)
    u = u0 + n * t
    cu, su = math.cos(u), math.sin(u)
    ci, si = math.cos(incl), math.sin(incl)
    co, so = math.cos(raan), math.sin(raan)
    p_i = radius * np.array([cu * co - su * ci * so, cu * so + su * ci * co, su * si])
    v_i = radius * n * np.array([-su * co - cu * ci * so, -su * so + cu * ci * co, cu * si])
    th = OMEGA_E * t
    c, s = math.cos(th), math.sin(th)
    rot = np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])
    p = rot @ p_i
    v = rot @ v_i - np.cross([0.0, 0.0, OMEGA_E], p)
    return p, v


@dataclasses.dataclass
class Formation:
    """Two receivers on one circular orbit, receiver 2 leading by sep_m of arc."""

    altitude_m: float = 550e3
    sep_m: float = 50e3
    incl_deg: float = 53.0
    raan_deg: float = 0.0
    u0_deg: float = 20.0
    t0_s: float = 0.0
    dt_s: float = 1.0

    @property
    def radius(self) -> float:
        return WGS84_A + self.altitude_m

    def states(self, t):
        """(p1, v1, p2, v2) in ECEF at absolute time t."""
        r = self.radius
        du = self.sep_m / r
        u0 = math.radians(self.u0_deg)
        inc = math.radians(self.incl_deg)
        raan = math.radians(self.raan_deg)
        p1, v1 = orbit_state_ecef(t, r, inc, raan, u0)
        p2, v2 = orbit_state_ecef(t, r, inc, raan, u0 + du)
        return p1, v1, p2, v2

    def ephemerides(self, k_steps):
        """double[K][12] = p1, v1, p2, v2 per step epoch t0 + k dt."""
        out = np.empty((k_steps, 12), dtype=np.float64)
        for k in range(k_steps):
            out[k] = np.concatenate(self.states(self.t0_s + k * self.dt_s))
        return out


def truth_delay_doppler(formation: Formation, t, p_e, fc_hz, h=1e-3):
    """Per receiver: delay range/c and Doppler -(d range/dt)/lambda.

    The range rate is a fourth-order central difference of the range along the
    propagated orbit, independent of any closed-form Doppler expression.
    """
    lam = C_LIGHT / fc_hz

    def ranges(tt):
        p1, _, p2, _ = formation.states(tt)
        return np.array([np.linalg.norm(p1 - p_e), np.linalg.norm(p2 - p_e)])

    r0 = ranges(t)
    rate = (-ranges(t + 2 * h) + 8 * ranges(t + h) - 8 * ranges(t - h) + ranges(t - 2 * h)) / (12 * h)
    return r0 / C_LIGHT, -rate / lam


def track_point(formation: Formation, t_mid, along_km, cross_km):
    """The point on the sphere of radius WGS84_A reached from the formation's
    sub-satellite point at t_mid by along_km along the track and cross_km
    across it (positive: the side of velocity x up), as (lat_deg, lon_deg)."""
    p1, v1, p2, v2 = formation.states(t_mid)
    pm, vm = 0.5 * (p1 + p2), 0.5 * (v1 + v2)
    g = pm / np.linalg.norm(pm)
    t = vm - np.dot(vm, g) * g
    t /= np.linalg.norm(t)
    x = np.cross(g, t)
    a = along_km * 1e3 / WGS84_A
    c = cross_km * 1e3 / WGS84_A
    e = math.cos(c) * (math.cos(a) * g + math.sin(a) * t) + math.sin(c) * x
    return math.degrees(math.asin(e[2])), math.degrees(math.atan2(e[1], e[0]))


def pick_emitter(rng, formation: Formation, t_mid, along_km=(-150.0, 150.0), cross_km=(150.0, 450.0)):
    """Seeded emitter site near the formation's ground track at t_mid.

    It is placed along-track within along_km of the formation's sub-satellite
    point and cross-track at a distance in cross_km on a seeded side, so its
    mirror image about the ground track lies at least 2*cross_km[0] away.
    Returns (lat_deg, lon_deg) of a point on the ellipsoid (h = 0).
    """
    p1, v1, p2, v2 = formation.states(t_mid)
    pm, vm = 0.5 * (p1 + p2), 0.5 * (v1 + v2)
    g = pm / np.linalg.norm(pm)
    t = vm - np.dot(vm, g) * g
    t /= np.linalg.norm(t)
    x = np.cross(g, t)
    a = rng.uniform(*along_km) * 1e3 / WGS84_A
    side = 1.0 if rng.uniform() < 0.5 else -1.0
    c = side * rng.uniform(*cross_km) * 1e3 / WGS84_A
    e = math.cos(c) * (math.cos(a) * g + math.sin(a) * t) + math.sin(c) * x
    lat = math.degrees(math.asin(e[2]))
    lon = math.degrees(math.atan2(e[1], e[0]))
    return lat, lon


# --------------------------------------------------------------------------
# waveforms (Sec. IV-A) — all unit power
# --------------------------------------------------------------------------
def chirp(t, bw_hz, period_s):
    """Eq. 12, repeated every period: exp(j2pi(B/(2T) t^2 - B/2 t)), t mod T."""
    tt = np.mod(t, period_s)
    return np.exp(2j * np.pi * (bw_hz / (2 * period_s) * tt * tt - 0.5 * bw_hz * tt))


def sawtooth(t, bw_hz, period_s):
    """Chirp for one period, then its conjugate for the next (period 2T)."""
    tt = np.mod(t, 2 * period_s)
    up = chirp(tt, bw_hz, period_s)
    return np.where(tt < period_s, up, np.conj(up))


def tone(t, f_hz=0.0):
    """A pure tone; at f = 0 it sits exactly on the carrier."""
    return np.exp(2j * np.pi * f_hz * np.asarray(t, dtype=np.float64))


def gold_code_prn1():
    """The 1023-chip C/A Gold code of GPS PRN 1 as +-1 (chip 0 -> +1): the
    product of two 10-stage maximal-length sequences, G1 with feedback
    polynomial 1 + x^3 + x^10 and G2 with 1 + x^2 + x^3 + x^6 + x^8 + x^9 +
    x^10, G2 read at the phase given by the xor of its stages 2 and 6; both
    registers start all ones."""
    g1 = [1] * 10
    g2 = [1] * 10
    out = np.empty(1023, dtype=np.int8)
    for k in range(1023):
        chip = g1[9] ^ g2[1] ^ g2[5]
        out[k] = 1 - 2 * chip
        f1 = g1[2] ^ g1[9]
        f2 = g2[1] ^ g2[2] ^ g2[5] ^ g2[7] ^ g2[8] ^ g2[9]
        g1 = [f1] + g1[:9]
        g2 = [f2] + g2[:9]
    return out


def gps_ca(t, code, bits, chip_rate_hz=1.023e6, bit_rate_hz=50.0):
    """BPSK spoofing waveform: the repeating 1 ms C/A code, rectangular chips,
    times a 50 bit/s navigation-data sequence (bits: +-1, indexed by
    whole bit periods from t = 0, wrapping)."""
    t = np.asarray(t, dtype=np.float64)
    chip = np.floor(t * chip_rate_hz).astype(np.int64) % code.size
    bit = np.floor(t * bit_rate_hz).astype(np.int64) % bits.size
    return (code[chip] * bits[bit]).astype(np.complex128)


def bandlimited_noise_spectrum(rng, n_fft, fs_hz, bw_hz):
    """Spectrum of a unit-power periodic complex Gaussian noise of two-sided
    bandwidth bw_hz (brick-wall mask), length n_fft samples at fs_hz."""
    f = np.fft.fftfreq(n_fft, 1.0 / fs_hz)
    mask = np.abs(f) <= 0.5 * bw_hz
    spec = (rng.standard_normal(n_fft) + 1j * rng.standard_normal(n_fft)) * mask
    p = np.sum(np.abs(spec) ** 2) / n_fft ** 2  # mean |x|^2 of the ifft
    return spec / math.sqrt(p), f


def delayed_noise(spec, f, delay_s, n_out):
    """x(n T_s - delay) for n < n_out, via a frequency-domain phase ramp on
    the periodic band-limited sequence defined by spec."""
    x = np.fft.ifft(spec * np.exp(-2j * np.pi * f * delay_s))
    return x[:n_out]


# --------------------------------------------------------------------------
# scene
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    fs_hz: float
    fc_hz: float
    n_samples: int
    k_steps: int
    fmt: str
    grid: dict
    ephem: np.ndarray          # (K, 12) float64
    y1: np.ndarray             # (K, N, 2) float32 / int16 / int8
    y2: np.ndarray
    emitter_lat_deg: float
    emitter_lon_deg: float
    emitter_ecef: np.ndarray
    tau: np.ndarray            # (K, 2) truth delays (s)
    fdop: np.ndarray           # (K, 2) truth Dopplers (Hz)
    meta: dict

    @property
    def G(self) -> int:
        return int(self.grid["nlat"]) * int(self.grid["nlon"])

    @property
    def fmt_code(self) -> int:
        return FORMAT_CODE[self.fmt]

    def y_complex(self, which: int) -> np.ndarray:
        """(K, N) complex128 view of receiver `which` (1 or 2), exact."""
        y = self.y1 if which == 1 else self.y2
        return y[..., 0].astype(np.float64) + 1j * y[..., 1].astype(np.float64)


def quantize(y, fmt, total_power):
    """Interleaved I/Q array (N, 2) in the storage format.

    ci16: each component scaled to a standard deviation of 2048 LSB, clipped
    at +-32767; ci8: 24 LSB, clipped at +-127; c64: float32 unscaled.
    """
    iq = np.stack([y.real, y.imag], axis=-1)
    if fmt == "c64":
        return iq.astype(np.float32)
    std = math.sqrt(total_power / 2.0)
    if fmt == "ci16":
        q = np.clip(np.rint(iq * (2048.0 / std)), -32767, 32767)
        return q.astype(np.int16)
    if fmt == "ci8":
        q = np.clip(np.rint(iq * (24.0 / std)), -127, 127)
        return q.astype(np.int8)
    raise ValueError(f"unknown format {fmt!r}")


def make_scene(
    *,
    seed: int,
    fs_hz: float,
    n_samples: int,
    k_steps: int,
    fmt: str,
    waveform: str,
    snr_db: float | None,
    grid_n: int | tuple,
    grid_spacing_m: float,
    fc_hz: float = 1575.42e6,
    bw_hz: float = 2e6,
    chirp_bw_hz: float = 10e6,
    chirp_period_s: float = 10e-6,
    tone_hz: float = 0.0,
    formation: Formation | None = None,
    integer_delays: bool = False,
    grid_offset_cells: tuple = (0, 0),
    emitter: tuple | None = None,
) -> Scene:
    """Build one seeded scene.

    snr_db=None gives noise-free captures. integer_delays=True rounds receiver
    1's delay to a whole sample and receiver 2's to receiver 1's plus the
    differential delay rounded to a whole sample (noise waveform only), so the
    true alignment is an exact integer lag. The grid is centred on the emitter
    unless grid_offset_cells moves its centre by whole cells (lat, lon).
    emitter = (lat_deg, lon_deg) places the emitter there instead of at a
    seeded site near the ground track.
    """
    rng = np.random.default_rng(seed)
    form = formation or Formation()
    t_mid = form.t0_s + 0.5 * (k_steps - 1) * form.dt_s
    lat_e, lon_e = pick_emitter(rng, form, t_mid) if emitter is None else emitter
    p_e = geodetic_to_ecef(lat_e, lon_e, 0.0)
    ephem = form.ephemerides(k_steps)
    nlat, nlon = (grid_n, grid_n) if isinstance(grid_n, int) else grid_n
    if grid_offset_cells != (0, 0):
        # centre moved by whole cells: spacing is metres on the ellipsoid at the
        # emitter latitude (meridian / prime-vertical radii)
        s = math.sin(math.radians(lat_e))
        w = math.sqrt(1.0 - WGS84_E2 * s * s)
        m_rad = WGS84_A * (1.0 - WGS84_E2) / w ** 3
        n_rad = WGS84_A / w
        dlat = math.degrees(grid_spacing_m / m_rad)
        dlon = math.degrees(grid_spacing_m / (n_rad * math.cos(math.radians(lat_e))))
        lat0 = lat_e - grid_offset_cells[0] * dlat
        lon0 = lon_e - grid_offset_cells[1] * dlon
    else:
        lat0, lon0 = lat_e, lon_e
    grid = dict(lat0_deg=lat0, lon0_deg=lon0, dlat_m=grid_spacing_m, dlon_m=grid_spacing_m,
                nlat=int(nlat), nlon=int(nlon))

    n = n_samples
    ts = 1.0 / fs_hz
    t_n = np.arange(n, dtype=np.float64) * ts
    amp = 1.0 if snr_db is None else math.sqrt(10.0 ** (snr_db / 10.0))
    noise_p = 0.0 if snr_db is None else 1.0
    y1 = np.empty((k_steps, n, 2), dtype={"c64": np.float32, "ci16": np.int16, "ci8": np.int8}[fmt])
    y2 = np.empty_like(y1)
    taus = np.empty((k_steps, 2))
    fds = np.empty((k_steps, 2))
    chirp_t0 = rng.uniform(0.0, chirp_period_s)
    if waveform == "gps_ca":
        code = gold_code_prn1()
        bits = rng.choice(np.array([-1, 1], dtype=np.int8), size=4096)
    for k in range(k_steps):
        tk = form.t0_s + k * form.dt_s
        tau, fd = truth_delay_doppler(form, tk, p_e, fc_hz)
        taus[k], fds[k] = tau, fd
        sig = []
        if waveform == "noise":
            n_fft = 1 << int(math.ceil(math.log2(2 * n + 8192)))
            spec, f = bandlimited_noise_spectrum(rng, n_fft, fs_hz, bw_hz)
            if integer_delays:
                d1 = int(np.rint(tau[0] * fs_hz))
                d2 = d1 + int(np.rint((tau[1] - tau[0]) * fs_hz))
                base = np.fft.ifft(spec)
                ref = d1
                sig = [np.roll(base, d - ref)[:n] for d in (d1, d2)]
            else:
                ref = tau[0]
                sig = [delayed_noise(spec, f, tau[i] - ref, n) for i in range(2)]
        elif waveform == "chirp":
            sig = [chirp(chirp_t0 + t_n - tau[i], chirp_bw_hz, chirp_period_s) for i in range(2)]
        elif waveform == "sawtooth":
            sig = [sawtooth(chirp_t0 + t_n - tau[i], chirp_bw_hz, chirp_period_s) for i in range(2)]
        elif waveform == "tone":
            sig = [tone(t_n - tau[i], tone_hz) for i in range(2)]
        elif waveform == "gps_ca":
            sig = [gps_ca(tk + t_n - tau[i], code, bits) for i in range(2)]
        else:
            raise ValueError(f"unknown waveform {waveform!r}")
        for i, dst in enumerate((y1, y2)):
            y = amp * sig[i] * np.exp(2j * np.pi * fd[i] * t_n)
            if noise_p > 0.0:
                y = y + (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * math.sqrt(0.5)
            dst[k] = quantize(y, fmt, amp * amp + noise_p)
    meta = dict(seed=seed, waveform=waveform, snr_db=snr_db, bw_hz=bw_hz, chirp_bw_hz=chirp_bw_hz,
                chirp_period_s=chirp_period_s, formation=dataclasses.asdict(form),
                integer_delays=integer_delays)
    return Scene(fs_hz=fs_hz, fc_hz=fc_hz, n_samples=n, k_steps=k_steps, fmt=fmt, grid=grid,
                 ephem=ephem, y1=y1, y2=y2, emitter_lat_deg=lat_e, emitter_lon_deg=lon_e,
                 emitter_ecef=p_e, tau=taus, fdop=fds, meta=meta)


def _cell_degrees(lat_deg, spacing_m):
    """Degrees of latitude and longitude spanned by one grid cell of
    spacing_m metres at lat_deg (meridian / prime-vertical radii)."""
    s = math.sin(math.radians(lat_deg))
    w = math.sqrt(1.0 - WGS84_E2 * s * s)
    m_rad = WGS84_A * (1.0 - WGS84_E2) / w ** 3
    n_rad = WGS84_A / w
    return math.degrees(spacing_m / m_rad), math.degrees(spacing_m / (n_rad * math.cos(math.radians(lat_deg))))


@dataclasses.dataclass
class Emitter:
    """One emitter of a multi-emitter scene: its node offset from the grid
    centre (cells, lat and lon), waveform and SNR (dB, per receiver sample,
    against the unit-power receiver noise)."""
    di: int
    dj: int
    waveform: str
    snr_db: float
    bw_hz: float = 2e6
    chirp_bw_hz: float | None = None      # None: the scene's chirp parameters
    chirp_period_s: float | None = None


@dataclasses.dataclass
class MultiScene:
    fs_hz: float
    fc_hz: float
    n_samples: int
    k_steps: int
    fmt: str
    grid: dict
    ephem: np.ndarray
    y1: np.ndarray
    y2: np.ndarray
    emitters: list             # [Emitter]
    emitter_nodes: list        # [(i, j)] grid node of each emitter
    emitter_latlon_deg: list   # [(lat, lon)]
    meta: dict

    @property
    def G(self) -> int:
        return int(self.grid["nlat"]) * int(self.grid["nlon"])

    @property
    def fmt_code(self) -> int:
        return FORMAT_CODE[self.fmt]


def make_multi_scene(
    *,
    seed: int,
    fs_hz: float,
    n_samples: int,
    k_steps: int,
    fmt: str,
    emitters: list,
    grid_n: int | tuple,
    grid_spacing_m: float,
    noise: bool = True,
    fc_hz: float = 1575.42e6,
    chirp_bw_hz: float = 10e6,
    chirp_period_s: float = 10e-6,
    formation: Formation | None = None,
) -> MultiScene:
    """Several stationary emitters transmitting at once (Sec. I: a crowded
    band where strong, weak and cyclostationary emitters share the
    receivers). Each emitter sits on a grid node (offset from the grid
    centre by whole cells); receiver i records the sum of every emitter's
    delayed, Doppler-shifted waveform (Eq. 1, one term per emitter) plus one
    unit-power noise. Waveforms are drawn independently per emitter.
    """
    rng = np.random.default_rng(seed)
    form = formation or Formation()
    t_mid = form.t0_s + 0.5 * (k_steps - 1) * form.dt_s
    lat0, lon0 = pick_emitter(rng, form, t_mid)
    dlat, dlon = _cell_degrees(lat0, grid_spacing_m)
    nlat, nlon = (grid_n, grid_n) if isinstance(grid_n, int) else grid_n
    ci, cj = (nlat - 1) // 2, (nlon - 1) // 2
    grid = dict(lat0_deg=lat0, lon0_deg=lon0, dlat_m=grid_spacing_m, dlon_m=grid_spacing_m,
                nlat=int(nlat), nlon=int(nlon))
    sites, nodes = [], []
    for e in emitters:
        if not (0 <= ci + e.di < nlat and 0 <= cj + e.dj < nlon):
            raise ValueError("emitter outside the grid")
        sites.append((lat0 + e.di * dlat, lon0 + e.dj * dlon))
        nodes.append((ci + e.di, cj + e.dj))
    p_e = [geodetic_to_ecef(la, lo, 0.0) for la, lo in sites]
    ephem = form.ephemerides(k_steps)
    n = n_samples
    t_n = np.arange(n, dtype=np.float64) / fs_hz
    amps = [math.sqrt(10.0 ** (e.snr_db / 10.0)) for e in emitters]
    noise_p = 1.0 if noise else 0.0
    cp = [(e.chirp_bw_hz or chirp_bw_hz, e.chirp_period_s or chirp_period_s) for e in emitters]
    chirp_t0 = [rng.uniform(0.0, p) for _, p in cp]
    code = gold_code_prn1()
    bits = [rng.choice(np.array([-1, 1], dtype=np.int8), size=4096) if e.waveform == "gps_ca" else None
            for e in emitters]
    dt = {"c64": np.float32, "ci16": np.int16, "ci8": np.int8}[fmt]
    y1 = np.empty((k_steps, n, 2), dtype=dt)
    y2 = np.empty_like(y1)
    for k in range(k_steps):
        tk = form.t0_s + k * form.dt_s
        acc = [np.zeros(n, np.complex128), np.zeros(n, np.complex128)]
        for m, e in enumerate(emitters):
            tau, fd = truth_delay_doppler(form, tk, p_e[m], fc_hz)
            if e.waveform == "noise":
                n_fft = 1 << int(math.ceil(math.log2(2 * n + 8192)))
                spec, f = bandlimited_noise_spectrum(rng, n_fft, fs_hz, e.bw_hz)
                sig = [delayed_noise(spec, f, tau[i] - tau[0], n) for i in range(2)]
            elif e.waveform == "chirp":
                sig = [chirp(chirp_t0[m] + t_n - tau[i], *cp[m]) for i in range(2)]
            elif e.waveform == "sawtooth":
                sig = [sawtooth(chirp_t0[m] + t_n - tau[i], *cp[m]) for i in range(2)]
            elif e.waveform == "tone":
                sig = [tone(t_n - tau[i]) for i in range(2)]
            elif e.waveform == "gps_ca":
                sig = [gps_ca(tk + t_n - tau[i], code, bits[m]) for i in range(2)]
            else:
                raise ValueError(f"waveform {e.waveform!r} not supported in a multi-emitter scene")
            for i in range(2):
                acc[i] += amps[m] * sig[i] * np.exp(2j * np.pi * fd[i] * t_n)
        total = sum(a * a for a in amps) + noise_p
        for i, dst in enumerate((y1, y2)):
            y = acc[i]
            if noise:
                y = y + (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * math.sqrt(0.5)
            dst[k] = quantize(y, fmt, total)
    meta = dict(seed=seed, emitters=[dataclasses.asdict(e) for e in emitters], noise=noise,
                formation=dataclasses.asdict(form))
    return MultiScene(fs_hz=fs_hz, fc_hz=fc_hz, n_samples=n, k_steps=k_steps, fmt=fmt, grid=grid,
                      ephem=ephem, y1=y1, y2=y2, emitters=list(emitters), emitter_nodes=nodes,
                      emitter_latlon_deg=sites, meta=meta)


def crowded(seed: int = 4, **kw) -> MultiScene:
    """Three emitters at once on a 121x121 grid at 1 km: two independent
    2 MHz noise emitters (one 3 dB weaker) and a 10 MHz / 10 us chirp;
    K=12 snapshots 15 s apart x N=16384 complex int16 at fs 12.5 MHz."""
    args = dict(seed=seed, fs_hz=12.5e6, n_samples=16384, k_steps=12, fmt="ci16", grid_n=121,
                grid_spacing_m=1000.0, formation=Formation(dt_s=15.0),
                emitters=[Emitter(0, 0, "noise", -3.0), Emitter(-25, 30, "chirp", -3.0),
                          Emitter(35, -20, "noise", -6.0)])
    args.update(kw)
    return make_multi_scene(**args)


def four_jammers(seed: int = 5, **kw) -> MultiScene:
    """The paper's capture scenario (Sec. IV-B) at full size: a GPS L1 C/A
    spoofer, a pure tone, a chirp (2 MHz, 20 us) and a sawtooth (200 kHz,
    5 ms) at equal power on the corners of a rectangle; 58 captures 1 s apart,
    each 50 ms at 5 MHz complex (N = 250000) on L1; a search grid of about
    4 deg of latitude by 9 deg of longitude (401 x 801 nodes at 1.1 km).
    The SNR (-10 dB per emitter) and the geometry are this simulator's."""
    args = dict(seed=seed, fs_hz=5e6, n_samples=250_000, k_steps=58, fmt="ci16", grid_n=(401, 801),
                grid_spacing_m=1100.0, formation=Formation(dt_s=1.0),
                emitters=[Emitter(-60, -150, "gps_ca", -10.0), Emitter(-60, 150, "tone", -10.0),
                          Emitter(60, -150, "chirp", -10.0, chirp_bw_hz=2e6, chirp_period_s=20e-6),
                          Emitter(60, 150, "sawtooth", -10.0, chirp_bw_hz=200e3, chirp_period_s=5e-3)])
    args.update(kw)
    return make_multi_scene(**args)


# --------------------------------------------------------------------------
# the workloads (sizes, formats, waveforms and SNRs of the five workloads)
# --------------------------------------------------------------------------
def learned(seed: int = 5, *, n_samples: int = 65536, k_steps: int = 20, footprint_m: float = 2.0e6,
            judge_spacing_m: float = 500.0, snr_db=(-21.0, -12.0), waveforms=("noise", "chirp", "gps_ca"),
            margin_m: float = 60e3, cross_km: float = 1200.0, fs_hz: float = 12.5e6) -> Scene:
    """One scene of the learned-proposal workload: a footprint_m square
    (lat/lon grid at judge_spacing_m, the full-grid search) centred cross_km
    from the ground track on the equator side, with the formation near the
    northern apex of its orbit (u0 = 86 deg), where the track runs east-west
    and the footprint lies wholly on one side of it (no mirror image inside).
    The emitter sits at a seeded point of the footprint (at least margin_m
    from its edges), with a seeded waveform and SNR (uniform in snr_db);
    K = 20 snapshots 1 s apart of N = 65536 complex int16 samples at
    12.5 MHz. The noise is 10 MHz wide; the chirp sweeps 10 MHz every 2 ms
    and the GPS C/A spoofer repeats every 1 ms, both longer than the
    footprint's delay span (a chirp repeating every 10 us would put a
    copy of the emitter's delay ridge every 125 lags)."""
    rng = np.random.default_rng(seed)
    form = Formation(u0_deg=86.0)
    t_mid = form.t0_s + 0.5 * (k_steps - 1) * form.dt_s
    north = track_point(form, t_mid, 0.0, 1.0)[0] > track_point(form, t_mid, 0.0, -1.0)[0]
    lat_c, lon_c = track_point(form, t_mid, 0.0, -cross_km if north else cross_km)
    half = 0.5 * footprint_m - margin_m
    di_m, dj_m = rng.uniform(-half, half), rng.uniform(-half, half)
    dlat, dlon = _cell_degrees(lat_c, 1.0)  # degrees per metre at the centre
    lat_e, lon_e = lat_c + di_m * dlat, lon_c + dj_m * dlon
    waveform = str(waveforms[int(rng.integers(len(waveforms)))])
    snr = float(rng.uniform(*snr_db)) if isinstance(snr_db, tuple) else float(snr_db)
    n_side = int(round(footprint_m / judge_spacing_m)) + 1
    sc = make_scene(seed=int(rng.integers(1 << 31)), fs_hz=fs_hz, n_samples=n_samples, k_steps=k_steps,
                    fmt="ci16", waveform=waveform, snr_db=snr, grid_n=n_side, grid_spacing_m=judge_spacing_m,
                    bw_hz=10e6, chirp_bw_hz=10e6, chirp_period_s=2e-3, formation=form,
                    emitter=(lat_e, lon_e))
    sc.grid = dict(lat0_deg=lat_c, lon0_deg=lon_c, dlat_m=judge_spacing_m, dlon_m=judge_spacing_m,
                   nlat=n_side, nlon=n_side)
    sc.meta.update(workload="learned", footprint_m=footprint_m, emitter_offset_m=(di_m, dj_m),
                   waveform=waveform, snr_db=snr)
    return sc


def tiny(seed: int = 1, **kw) -> Scene:
    """101x101 grid at 1 km, K=1 x N=4096 complex64, 2 MHz noise, fs 5 MHz, -5 dB."""
    args = dict(seed=seed, fs_hz=5e6, n_samples=4096, k_steps=1, fmt="c64", waveform="noise",
                snr_db=-5.0, grid_n=101, grid_spacing_m=1000.0, bw_hz=2e6)
    args.update(kw)
    return make_scene(**args)


def mid(seed: int = 2, **kw) -> Scene:
    """1001x1001 grid at 100 m, K=20 x N=65536 complex int16, chirp 10 MHz / 10 us,
    fs 12.5 MHz, -15 dB."""
    args = dict(seed=seed, fs_hz=12.5e6, n_samples=65536, k_steps=20, fmt="ci16", waveform="chirp",
                snr_db=-15.0, grid_n=1001, grid_spacing_m=100.0, chirp_bw_hz=10e6,
                chirp_period_s=10e-6)
    args.update(kw)
    return make_scene(**args)


def large(seed: int = 3, **kw) -> Scene:
    """4001x4001 grid at 400 m, K=50 x N=131072 complex int8, 18 MHz noise,
    fs 20 MHz, -20 dB."""
    args = dict(seed=seed, fs_hz=20e6, n_samples=131072, k_steps=50, fmt="ci8", waveform="noise",
                snr_db=-20.0, grid_n=4001, grid_spacing_m=400.0, bw_hz=18e6)
    args.update(kw)
    return make_scene(**args)


WORKLOADS = {"tiny": tiny, "mid": mid, "large": large}
LEARNED = learned
MULTI_WORKLOADS = {"crowded": crowded, "four_jammers": four_jammers}
