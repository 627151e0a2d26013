"""The C ABI without a GPU: the library builds, loads, exports every function
include/dg.h declares, the ctypes layouts match the C layouts, and argument
validation reports errors through the ABI before touching the device."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dg.h")


@pytest.fixture(scope="module")
def P():
    from paper_2508_06672_gb300 import build

    build.build()
    import paper_2508_06672_gb300 as P

    return P


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(dg_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_function_is_exported(P):
    names = declared_functions()
    assert len(names) >= 14
    L = P.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(P.EXPORTED_SYMBOLS)
    out = subprocess.run(["nm", "-D", "--defined-only", P.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dg_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_c(P):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "dg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dg_grid), sizeof(dg_ephem),
         sizeof(dg_options), sizeof(dg_fix), offsetof(dg_fix, refine_n), offsetof(dg_fix, refined_lat_deg),
         offsetof(dg_fix, sub_lat_deg), sizeof(dg_coarse_step), offsetof(dg_coarse_step, mu),
         offsetof(dg_options, timing), offsetof(dg_options, tiles), sizeof(dg_peak), offsetof(dg_peak, lat_deg),
         sizeof(dg_tuning), offsetof(dg_tuning, ms), offsetof(dg_tuning, cached));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(P.dg_grid), C.sizeof(P.dg_ephem), C.sizeof(P.dg_options), C.sizeof(P.dg_fix),
            P.dg_fix.refine_n.offset, P.dg_fix.refined_lat_deg.offset, P.dg_fix.sub_lat_deg.offset,
            C.sizeof(P.dg_coarse_step), P.dg_coarse_step.mu.offset, P.dg_options.timing.offset,
            P.dg_options.tiles.offset, C.sizeof(P.dg_peak), P.dg_peak.lat_deg.offset, C.sizeof(P.dg_tuning),
            P.dg_tuning.ms.offset, P.dg_tuning.cached.offset]
    assert vals == want


def test_abi_version_and_defaults(P):
    assert P.dg_abi_version() == 1
    o = P.dg_options_default()
    assert (o.delay, o.acc, o.prec, o.algo, o.row0, o.nrows, o.timing) == (0, 0, 0, 0, 0, 0, 0)


GOOD = dict(lat0_deg=10.0, lon0_deg=20.0, dlat_m=100.0, dlon_m=100.0, nlat=3, nlon=3)


@pytest.mark.parametrize("patch,K,fs,fc", [
    (dict(nlat=0), 1, 5e6, 1.5e9),
    (dict(dlat_m=-1.0), 1, 5e6, 1.5e9),
    (dict(lat0_deg=float("nan")), 1, 5e6, 1.5e9),
    (dict(lat0_deg=89.5), 1, 5e6, 1.5e9),
    ({}, 0, 5e6, 1.5e9),
    ({}, 1, 0.0, 1.5e9),
    ({}, 1, 5e6, -1.0),
])
def test_create_rejects_bad_arguments(P, patch, K, fs, fc):
    grid = dict(GOOD, **patch)
    with pytest.raises(P.DGError) as e:
        P.dg_create(grid, np.ones((max(K, 1), 12)), K, fs, fc)
    assert e.value.status == P.DG_EINVAL
    assert P.dg_last_error(None)


def test_create_rejects_bad_options_and_ephemerides(P):
    o = P.dg_options_default()
    o.delay = 7
    with pytest.raises(P.DGError) as e:
        P.dg_create(GOOD, np.ones((1, 12)), 1, 5e6, 1.5e9, o)
    assert e.value.status == P.DG_EINVAL and "delay" in P.dg_last_error(None)
    o = P.dg_options_default()
    o.row0, o.nrows = 2, 5
    with pytest.raises(P.DGError):
        P.dg_create(GOOD, np.ones((1, 12)), 1, 5e6, 1.5e9, o)
    eph = np.ones((2, 12))
    eph[1, 4] = np.inf
    with pytest.raises(P.DGError) as e:
        P.dg_create(GOOD, eph, 2, 5e6, 1.5e9)
    assert "ephemeris 1" in P.dg_last_error(None)


def test_null_context_calls_fail_cleanly(P):
    assert P.lib().dg_cost_surface(None, None) == P.DG_EINVAL
    assert P.lib().dg_sync(None) == P.DG_EINVAL
    assert P.lib().dg_destroy(None) == P.DG_OK
    assert P.dg_launch_count(None) == -1


def test_binding_has_no_cpu_fallback(P):
    """The binding and the package import nothing from the oracle or the
    input generator, so no product call can route through them."""
    pkg = os.path.join(ROOT, "paper_2508_06672_gb300")
    for name in os.listdir(pkg):
        if not name.endswith(".py"):
            continue
        for line in open(os.path.join(pkg, name)):
            words = line.split()
            if words[:1] in (["import"], ["from"]):
                mod = words[1].split(".")[0]
                assert mod not in ("oracle", "sim"), (name, line)
