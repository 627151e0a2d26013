"""Python access to the plain FP64 CPU oracle (``dg_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package. The CUDA
library and its Python binding never do.

``build()`` compiles ``dg_oracle.c`` with gcc (OpenMP, ``-ffp-contract=off``)
into ``oracle/_build/``; the functions below marshal numpy arrays into it.
Parity status of each function is recorded in its pins under ``tests/``.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libdg_oracle.so")
_LOCK = threading.Lock()
_LIB = None


class Grid(C.Structure):
    _fields_ = [("lat0_deg", C.c_double), ("lon0_deg", C.c_double), ("dlat_m", C.c_double),
                ("dlon_m", C.c_double), ("nlat", C.c_int32), ("nlon", C.c_int32)]

    @classmethod
    def from_dict(cls, d):
        return cls(float(d["lat0_deg"]), float(d["lon0_deg"]), float(d["dlat_m"]),
                   float(d["dlon_m"]), int(d["nlat"]), int(d["nlon"]))


def build(force: bool = False, src: str = _SRC, out: str = _OUT) -> str:
    """Compile an oracle source (default: dg_oracle.c) if missing or stale."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _bind(path):
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    L.dgo_geodetic_to_ecef.argtypes = [C.c_double, C.c_double, C.c_double, dp]
    L.dgo_grid_step_rad.argtypes = [C.POINTER(Grid), dp, dp]
    L.dgo_grid_node.argtypes = [C.POINTER(Grid), C.c_int64, C.c_int64, dp, dp]
    L.dgo_grid_ecef.argtypes = [C.POINTER(Grid), dp]
    L.dgo_geometry.argtypes = [dp, dp, C.c_double, C.c_double, dp]
    L.dgo_lagrange4.argtypes = [C.c_double, dp]
    L.dgo_correlate.argtypes = [dp, dp, C.c_int64, C.c_double, C.c_double, C.c_int, dp]
    L.dgo_cost_points.argtypes = [C.POINTER(Grid), dp, C.c_int32, C.c_double, C.c_double,
                                  dp, dp, C.c_int64, C.c_int, C.c_int,
                                  C.POINTER(C.c_int64), C.c_int64, dp, dp, dp, C.c_int]
    L.dgo_cost_points.restype = C.c_int
    L.dgo_node_geometry.argtypes = [C.POINTER(Grid), dp, C.c_int32, C.c_double, C.c_double, dp, dp]
    L.dgo_node_geometry.restype = C.c_int
    L.dgo_argmax.argtypes = [dp, C.c_int64]
    L.dgo_argmax.restype = C.c_int64
    L.dgo_detect.argtypes = [dp, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_int64, C.POINTER(C.c_int64)]
    L.dgo_detect.restype = C.c_int64
    return L


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _bind(build())
    return _LIB


@contextlib.contextmanager
def using(path):
    """Route this module's functions to another build of an oracle source.

    The mutation tests plant one mistake in a copy of dg_oracle.c, build it,
    and run the pins through this to check that some pin catches it."""
    global _LIB
    lib()
    alt = _bind(path)
    with _LOCK:
        prev, _LIB = _LIB, alt
    try:
        yield
    finally:
        with _LOCK:
            _LIB = prev


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def iq_to_f64(y):
    """(…, N, 2) interleaved I/Q of any storage type -> float64, exactly."""
    return _f64c(np.asarray(y).astype(np.float64))


def geodetic_to_ecef(lat_rad, lon_rad, h=0.0):
    out = np.empty(3)
    lib().dgo_geodetic_to_ecef(float(lat_rad), float(lon_rad), float(h), _dp(out))
    return out


def grid_step_rad(grid):
    a, b = C.c_double(), C.c_double()
    lib().dgo_grid_step_rad(C.byref(Grid.from_dict(grid)), C.byref(a), C.byref(b))
    return a.value, b.value


def grid_node(grid, i, j):
    a, b = C.c_double(), C.c_double()
    lib().dgo_grid_node(C.byref(Grid.from_dict(grid)), int(i), int(j), C.byref(a), C.byref(b))
    return a.value, b.value


def grid_ecef(grid):
    g = Grid.from_dict(grid)
    out = np.empty((g.nlat * g.nlon, 3))
    lib().dgo_grid_ecef(C.byref(g), _dp(out))
    return out


def geometry(pc, eph, fs, fc):
    """-> (dtau s, dfreq Hz, D samples, nu cycles/sample)."""
    out = np.empty(4)
    lib().dgo_geometry(_dp(_f64c(pc)), _dp(_f64c(eph)), float(fs), float(fc), _dp(out))
    return tuple(out)


def lagrange4(mu):
    out = np.empty(4)
    lib().dgo_lagrange4(float(mu), _dp(out))
    return out


def correlate(y1, y2, D, nu, delay_mode=0):
    """Complex C of Eq. 11 for one (candidate, snapshot); y1/y2 complex or (N, 2)."""
    y1 = np.asarray(y1)
    y2 = np.asarray(y2)
    if np.iscomplexobj(y1):
        y1 = np.stack([y1.real, y1.imag], -1)
    if np.iscomplexobj(y2):
        y2 = np.stack([y2.real, y2.imag], -1)
    a, b = iq_to_f64(y1), iq_to_f64(y2)
    if a.shape != b.shape or a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("y1, y2 must both be (N, 2)")
    out = np.empty(2)
    lib().dgo_correlate(_dp(a), _dp(b), a.shape[0], float(D), float(nu), int(delay_mode), _dp(out))
    return complex(out[0], out[1])


def cost_points(grid, ephem, fs, fc, y1, y2, idx, delay_mode=0, acc_mode=0, nthreads=0,
                want_corr=False, want_geom=False):
    """Cost at selected candidates (linear indices). y1/y2 are (K, N, 2).

    Returns cost (npts,) and, if asked, C_k (npts, K) complex and the
    geometry (npts, K, 4)."""
    eph = _f64c(ephem)
    a, b = iq_to_f64(y1), iq_to_f64(y2)
    K, N = a.shape[0], a.shape[1]
    if eph.shape != (K, 12) or b.shape != a.shape:
        raise ValueError("shape mismatch")
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    cost = np.empty(idx.size)
    corr = np.empty((idx.size, K, 2)) if want_corr else None
    geom = np.empty((idx.size, K, 4)) if want_geom else None
    rc = lib().dgo_cost_points(C.byref(Grid.from_dict(grid)), _dp(eph), K, float(fs), float(fc),
                               _dp(a), _dp(b), N, int(delay_mode), int(acc_mode),
                               idx.ctypes.data_as(C.POINTER(C.c_int64)), idx.size, _dp(cost),
                               _dp(corr) if corr is not None else None,
                               _dp(geom) if geom is not None else None, int(nthreads))
    if rc != 0:
        raise ValueError("dgo_cost_points rejected its arguments")
    out = [cost]
    if want_corr:
        out.append(corr[..., 0] + 1j * corr[..., 1])
    if want_geom:
        out.append(geom)
    return out[0] if len(out) == 1 else tuple(out)


def cost_surface(grid, ephem, fs, fc, y1, y2, delay_mode=0, acc_mode=0, nthreads=0, rows=None):
    """Whole cost surface (nlat, nlon), or rows [r0, r1) of it."""
    nlat, nlon = int(grid["nlat"]), int(grid["nlon"])
    r0, r1 = (0, nlat) if rows is None else rows
    idx = np.arange(r0 * nlon, r1 * nlon, dtype=np.int64)
    c = cost_points(grid, ephem, fs, fc, y1, y2, idx, delay_mode, acc_mode, nthreads)
    return c.reshape(r1 - r0, nlon)


def node_geometry(grid, ephem, fs, fc):
    """Eq. 3-10 at every node: D (K, nlat, nlon) in samples and nu (K, nlat,
    nlon) in cycles per sample."""
    g = Grid.from_dict(grid)
    eph = _f64c(ephem).reshape(-1, 12)
    K = eph.shape[0]
    D = np.empty((K, g.nlat, g.nlon))
    nu = np.empty((K, g.nlat, g.nlon))
    if lib().dgo_node_geometry(C.byref(g), _dp(eph), K, float(fs), float(fc), _dp(D), _dp(nu)) != 0:
        raise MemoryError("dgo_node_geometry")
    return D, nu


def argmax(cost):
    c = _f64c(np.ravel(cost))
    return int(lib().dgo_argmax(_dp(c), c.size))


def detect(cost, threshold, radius, max_peaks=64):
    """Threshold detection on a surface (nlat, nlon): linear indices of the
    peaks, strongest first."""
    c = _f64c(cost)
    if c.ndim != 2:
        raise ValueError("cost must be (nlat, nlon)")
    out = np.empty(max(1, int(max_peaks)), dtype=np.int64)
    n = lib().dgo_detect(_dp(c), c.shape[0], c.shape[1], float(threshold), int(radius), int(max_peaks),
                         out.ctypes.data_as(C.POINTER(C.c_int64)))
    if n < 0:
        raise MemoryError("dgo_detect")
    return out[:n].copy()


def parabola_offset(a, b, d):
    """Vertex of the parabola through (-1, a), (0, b), (1, d), in nodes:
    0.5 (a - d) / (a - 2 b + d) where that curvature is negative (kept within
    [-0.5, 0.5]), else 0 (not in the paper: a sub-node estimate reported
    beside the grid maximum)."""
    den = (a - 2.0 * b) + d
    if not (den < 0.0):
        return 0.0
    x = 0.5 * (a - d) / den
    return 0.0 if x != x else min(0.5, max(-0.5, x))


def subcell(cost, i, j):
    """(di, dj): the parabolic offsets of node (i, j) of a surface (nlat, nlon)
    along rows and columns; 0 at an edge or with a non-finite neighbour."""
    c = np.asarray(cost, dtype=np.float64)
    n0, n1 = c.shape
    di = parabola_offset(c[i - 1, j], c[i, j], c[i + 1, j]) if 0 < i < n0 - 1 else 0.0
    dj = parabola_offset(c[i, j - 1], c[i, j], c[i, j + 1]) if 0 < j < n1 - 1 else 0.0
    if not np.all(np.isfinite([c[max(i - 1, 0), j], c[min(i + 1, n0 - 1), j]])):
        di = 0.0
    if not np.all(np.isfinite([c[i, max(j - 1, 0)], c[i, min(j + 1, n1 - 1)]])):
        dj = 0.0
    return di, dj


def refine_grid(grid, index, spacing_m, window_m):
    """Local grid for dense re-evaluation around a coarse cell (Algorithm 1's
    search repeated on a finer lattice): centred on the cell's latitude and
    longitude, spacing_m apart in metres at that latitude (the grid reading of
    Sec. III), with round(window_m / spacing_m) nodes on each side of the
    centre, rounded half away from zero like the lag of Eq. 9."""
    nlon = int(grid["nlon"])
    lat, lon = grid_node(grid, index // nlon, index % nlon)
    half = int(np.floor(window_m / spacing_m + 0.5))
    return dict(lat0_deg=np.degrees(lat), lon0_deg=np.degrees(lon), dlat_m=float(spacing_m),
                dlon_m=float(spacing_m), nlat=2 * half + 1, nlon=2 * half + 1)


def scene_args(scene):
    """(grid, ephem, fs, fc, y1, y2) of a sim.Scene."""
    return scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz, scene.y1, scene.y2
