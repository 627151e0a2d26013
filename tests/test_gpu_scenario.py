"""The paper's capture scenario (Sec. IV-B) at full size on the device: a
GPS L1 C/A spoofer, a tone, a chirp and a sawtooth jammer at equal power,
58 captures of 50 ms at 5 MHz, 1 s apart, over a ~4 x 9 degree grid.

Checks the qualitative results the paper reports for it: after summing the
58 snapshot grids the surface holds one sharp peak per emitter at its true
position and nothing else above half the maximum, while a single snapshot
is ambiguous (strong peaks away from every emitter). Device values are
compared with the oracle at the emitters and at sampled nodes."""
import numpy as np
import pytest

import oracle
import sim
from gpu_common import package, rel_err, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    return sim.four_jammers()


def _surface(scene, k=None, **opts):
    torch = torch_cuda()
    P = package()
    eph, y1, y2 = scene.ephem, scene.y1, scene.y2
    if k is not None:
        eph, y1, y2 = eph[k:k + 1], y1[k:k + 1], y2[k:k + 1]
    g = P.Geolocator(scene.grid, eph, scene.fs_hz, scene.fc_hz, acc="mag", **opts)
    g.load_captures(scene.fmt, torch.from_numpy(y1).cuda(), torch.from_numpy(y2).cuda())
    return g, g.cost_surface()


def _far(p, nodes, d):
    return all(max(abs(p["i"] - i), abs(p["j"] - j)) > d for i, j in nodes)


@pytest.mark.parametrize("opts", [dict(), dict(algo="cdft", contract="fp16x3")],
                         ids=["direct", "cdft_fp16x3_auto_chunk"])
def test_four_jammers_accumulated(scene, opts):
    g, c = _surface(scene, **opts)
    nlon = scene.grid["nlon"]
    peaks = g.detect(c, 0.5, relative=True, radius=5, max_peaks=16)
    if "algo" in opts:
        # the ~900 km wide grid spans a wide FDOA range: the automatic chunk
        # is short enough for the interpolation bound (and at most 2048 on
        # the tensor cores)
        lo, hi = g.cdft_chunks()
        assert 64 <= lo <= hi <= 2048
    assert sorted((p["i"], p["j"]) for p in peaks) == sorted(scene.emitter_nodes)
    # sampled parity with the oracle: the emitters' nodes plus seeded random nodes
    rng = np.random.default_rng(7)
    idx = np.concatenate([[i * nlon + j for i, j in scene.emitter_nodes],
                          rng.choice(scene.G, size=28, replace=False)])
    ref = oracle.cost_points(*oracle.scene_args(scene), idx=idx, acc_mode=1)
    got = c.double().cpu().numpy().ravel()[idx]
    tol = 1e-4 if "algo" not in opts else 2e-4
    assert rel_err(got[:4], ref[:4]) < tol
    # away from the peaks |C| is a noise-like sum: compare against the
    # surface scale (error normalised by the mean value)
    assert np.max(np.abs(got - ref)) / np.mean(ref) < 5 * tol
    g.close()


def test_single_snapshot_is_ambiguous(scene):
    """One snapshot: the tone's streak and the chirp's repeated peaks put
    strong maxima far from every emitter."""
    g, c = _surface(scene, k=0)
    peaks = g.detect(c, 0.5, relative=True, radius=5, max_peaks=64)
    assert len(peaks) > 4
    assert any(_far(p, scene.emitter_nodes, 20) for p in peaks)
    g.close()
