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


def rel_err(gpu, ref, floor_frac=0.0, strong_frac=0.1):
    """max_p |gpu - ref| / (ref + floor_frac * mean(ref)); points where the
    reference is exactly zero (no overlap of the captures at that lag) must be
    exactly zero on the device too (else the error is infinite).

    With a floor (surfaces of one to a few snapshots, whose values can come
    arbitrarily close to zero), the result is also at least the plain
    pointwise error max |gpu - ref| / ref over the nodes at or above
    strong_frac of the maximum, so the floor loosens nothing there."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    zero = ref == 0
    if np.any(gpu[zero] != 0):
        return float("inf")
    if np.all(zero):
        return 0.0
    den = ref[~zero] + floor_frac * float(np.mean(ref))
    err = float(np.max(np.abs(gpu[~zero] - ref[~zero]) / den))
    if floor_frac > 0:
        strong = ref >= strong_frac * float(np.max(ref))
        strong &= ~zero
        err = max(err, float(np.max(np.abs(gpu[strong] - ref[strong]) / ref[strong])))
    return err


# (test, gap, tol, decisive) of every argmax comparison in this session; the
# conftest prints them at the end of the run
ARGMAX_RECORD = []


def _current_test():
    import os

    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def assert_argmax_consistent(gpu, ref, tol, near_tie=False):
    """Argmax of the device surface against the oracle's (ties to the lowest
    index on both sides).

    The oracle's relative gap between its two largest values is recorded and
    printed. Where it exceeds twice the error bound, the indices must be
    identical. Otherwise the seed is a near-tie: the caller must declare it
    (near_tie=True; an undeclared near-tie fails, and so does a declared one
    that is not), and the device's maximum must then be a valid maximum,
    within twice the bound of the oracle's largest value."""
    gpu = np.asarray(gpu).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    am_ref = oracle.argmax(ref)
    am_gpu = int(np.argmax(gpu))
    srt = np.sort(ref)[::-1]
    gap = 1.0 if srt.size < 2 else float((srt[0] - srt[1]) / srt[0])
    decisive = gap > 2 * tol
    ARGMAX_RECORD.append((_current_test(), gap, tol, decisive))
    print(f"argmax: oracle top-two gap {gap:.3e} (bound {tol:g}): "
          f"{'decisive' if decisive else 'near-tie'}; device {am_gpu}, oracle {am_ref}")
    if decisive:
        assert not near_tie, f"declared a near-tie, but the gap {gap:.3e} exceeds 2 x {tol:g}"
        assert am_gpu == am_ref, (am_gpu, am_ref)
    else:
        assert near_tie, f"undeclared near-tie: top-two gap {gap:.3e} is within 2 x {tol:g}"
        assert ref[am_gpu] >= srt[0] * (1 - 2 * tol), (am_gpu, am_ref, ref[am_gpu] / srt[0])
    return am_ref


def assert_global_argmax(scene, dev, tol, near_tie=False, max_nodes=4096):
    """The full-size argmax check, complete under the pointwise bound.

    If every node satisfies |dev - ref| <= tol * ref (the bound the sampled
    nodes are held to), a node q can hold the oracle's maximum only if
    dev[q] >= M (1 - tol) / (1 + tol), where M is the device's maximum: any
    other node has ref[q] <= dev[q] / (1 - tol) < M / (1 + tol), which is at
    most the oracle's value at the device's argmax. So the oracle evaluates
    exactly that set (a few nodes to a few hundred), the bound is checked on
    it, and the device's argmax must be the oracle's maximum over it (ties to
    the lowest index), or, for a declared near-tie, within twice the bound of
    it. Returns the device's argmax."""
    c = np.asarray(dev, dtype=np.float64).ravel()
    am = int(np.argmax(c))
    thr = c[am] * (1.0 - tol) / (1.0 + tol)
    cand = np.flatnonzero(c >= thr)
    assert am in cand and cand.size <= max_nodes, cand.size
    ref = oracle.cost_points(*oracle.scene_args(scene), idx=cand)
    ok = ~lag_boundary_mask(scene, cand)
    assert rel_err(c[cand][ok], ref[ok]) < tol
    print(f"global argmax: {cand.size} node(s) within reach of the device maximum {am}")
    pos = assert_argmax_consistent(c[cand], ref, tol, near_tie)
    if not near_tie:
        assert int(cand[pos]) == am
    return am
