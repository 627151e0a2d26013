"""dg_cost_surface_noalloc: the cost surface for callers that may not allocate
device memory while processing (it uses the library's static scratch array).

Called through the C ABI and compared with the allocating entry points
(dg_create / dg_load_capture / dg_cost_surface) on two calls in a row with
different problems, so that anything left behind in the shared scratch by the
first call would show in the second. Collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import sim
from gpu_common import package, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
FP64_TOL = 1e-9


def _reference(P, s, prec):
    torch = torch_cuda()
    with P.Geolocator(s.grid, s.ephem, s.fs_hz, s.fc_hz, prec=prec) as g:
        g.load_captures(s.fmt, torch.from_numpy(s.y1).cuda(), torch.from_numpy(s.y2).cuda())
        c = g.cost_surface()
        g.sync()
        return c.double().cpu().numpy()


def _noalloc(P, s, prec):
    torch = torch_cuda()
    y1 = torch.from_numpy(np.ascontiguousarray(s.y1)).cuda()
    y2 = torch.from_numpy(np.ascontiguousarray(s.y2)).cuda()
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = torch.full((s.grid["nlat"], s.grid["nlon"]), float("nan"), dtype=dt, device="cuda")
    opt = P.dg_options_default()
    opt.prec = P.DG_PREC_FP64 if prec == "fp64" else P.DG_PREC_FP32
    torch.cuda.synchronize()
    P.dg_cost_surface_noalloc(s.grid, s.ephem, s.fs_hz, s.fc_hz, s.fmt_code, y1.data_ptr(), y2.data_ptr(),
                              s.n_samples, out.data_ptr(), opt, torch.cuda.current_stream().cuda_stream)
    return out.double().cpu().numpy()


def test_noalloc_matches_allocating_path_on_two_calls_in_a_row():
    P = package()
    a = sim.make_scene(seed=31, fs_hz=12.5e6, n_samples=4096, k_steps=3, fmt="ci16", waveform="chirp",
                       snr_db=-5.0, grid_n=(41, 37), grid_spacing_m=150.0)
    b = sim.make_scene(seed=32, fs_hz=5e6, n_samples=2049, k_steps=2, fmt="c64", waveform="noise",
                       snr_db=0.0, grid_n=(23, 29), grid_spacing_m=900.0)
    for s, prec, tol, floor in ((a, "fp32", FP32_TOL, 0.01), (b, "fp64", FP64_TOL, 0.0)):
        got = _noalloc(P, s, prec)
        want = _reference(P, s, prec)
        assert np.all(np.isfinite(got))
        assert rel_err(got, want, floor) < tol, prec


def test_noalloc_rejects_problems_beyond_its_scratch():
    P = package()
    torch = torch_cuda()
    s = sim.make_scene(seed=33, fs_hz=5e6, n_samples=64, k_steps=4, fmt="c64", waveform="noise",
                       snr_db=0.0, grid_n=(1001, 1001), grid_spacing_m=100.0)
    y = torch.zeros((4 * 64, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros((1001, 1001), dtype=torch.float32, device="cuda")
    with pytest.raises(P.DGError) as e:
        P.dg_cost_surface_noalloc(s.grid, s.ephem, s.fs_hz, s.fc_hz, P.DG_IQ_C64, y.data_ptr(), y.data_ptr(),
                                  64, out.data_ptr())
    assert e.value.status == P.DG_EINVAL
    assert "static scratch holds" in str(e.value)
    assert bool(torch.all(out == 0))
