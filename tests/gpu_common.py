"""Shared helpers for the GPU parity tests (CUDA library vs CPU oracle)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def package():
    """The binding; builds the library first if it is missing."""
    import paper_2508_06672_gb300 as P
    import os

    if not os.path.exists(P.library_path()):
        from paper_2508_06672_gb300 import build

        build.build()
    return P


def gpu_surface(scene, **opts):
    """Run the library on a sim.Scene; returns (Geolocator, surface as numpy)."""
    torch = torch_cuda()
    P = package()
    g = P.Geolocator(scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz, **opts)
    g.load_captures(scene.fmt, torch.from_numpy(scene.y1).cuda(), torch.from_numpy(scene.y2).cuda())
    c = g.cost_surface()
    g.sync()
    return g, c.double().cpu().numpy()


def oracle_surface(scene, delay_mode=0, acc_mode=0, rows=None):
    return oracle.cost_surface(*oracle.scene_args(scene), delay_mode=delay_mode, acc_mode=acc_mode,
                               rows=rows)


def lag_boundary_mask(scene, idx, delay_mode=0, eps=1e-9):
    """Candidates whose lag decision sits within eps of a rounding boundary at
    some snapshot (|frac(D) - 0.5| < eps for round, |frac(D)| < eps for floor):
    there the last-ulp differences of the two sides' sin/cos in the geodetic
    conversion may legitimately pick the neighbouring lag."""
    _, geom = oracle.cost_points(*oracle.scene_args(scene), idx=np.asarray(idx), want_geom=True,
                                 delay_mode=delay_mode)
    D = geom[..., 2]
    fr = D - np.floor(D)
    near = np.abs(fr - 0.5) < eps if delay_mode == 0 else np.minimum(fr, 1 - fr) < eps
    return near.any(axis=1)


def rel_err(gpu, ref, floor_frac=0.0):
    """max_p |gpu - ref| / (ref + floor_frac * mean(ref)); points where the
    reference is exactly zero (no overlap of the captures at that lag) must be
    exactly zero on the device too (else the error is infinite)."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    zero = ref == 0
    if np.any(gpu[zero] != 0):
        return float("inf")
    if np.all(zero):
        return 0.0
    den = ref[~zero] + floor_frac * float(np.mean(ref))
    return float(np.max(np.abs(gpu[~zero] - ref[~zero]) / den))


def assert_argmax_consistent(gpu, ref, tol):
    """Argmax identity where the oracle's top two differ by more than the
    error bound; otherwise (a near-tie) the device's maximum must be a valid
    maximum: within 2 tol of the oracle's maximum value."""
    gpu = np.asarray(gpu).ravel()
    ref = np.asarray(ref).ravel()
    am_ref = oracle.argmax(ref)
    am_gpu = int(np.argmax(gpu))
    srt = np.sort(ref)[::-1]
    if srt[0] - srt[1] > 2 * tol * srt[0]:
        assert am_gpu == am_ref, (am_gpu, am_ref)
    else:
        assert ref[am_gpu] >= srt[0] * (1 - 2 * tol), (am_gpu, am_ref, ref[am_gpu] / srt[0])
    return am_ref
