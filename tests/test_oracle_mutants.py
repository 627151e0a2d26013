"""Plant one plausible mistake at a time in a copy of the oracle source and
check that at least one pin catches it. CPU only; the oracle itself is not
modified."""
import os
import shutil
import tempfile

import pytest

import oracle
import oracle_pins

# (name, text in dg_oracle.c, replacement) -- each text occurs exactly once
MUTANTS = [
    ("doppler_sign", "double f1 = -((r1x", "double f1 = ((r1x"),
    ("eq9_divides_by_fs", "out[2] = dtau * fs;", "out[2] = dtau / fs;"),
    ("tdoa_order", "double dtau = (rho2 - rho1)", "double dtau = (rho1 - rho2)"),
    ("range_drops_z", "double rho2 = sqrt((r2x * r2x + r2y * r2y) + r2z * r2z);",
     "double rho2 = sqrt(r2x * r2x + r2y * r2y);"),
    ("range_vector_sign", "double r1x = p1[0] - pc[0]", "double r1x = pc[0] - p1[0]"),
    ("ellipsoid_z", "out[2] = (n * (1.0 - e2) + h) * s;", "out[2] = (n + h) * s;"),
    ("grid_centre", "((double)i - 0.5 * (double)(g->nlat - 1))", "((double)i - 0.5 * (double)g->nlat)"),
    ("meridian_radius", "double m = DGO_WGS84_A * (1.0 - e2) / (w * w * w);", "double m = DGO_WGS84_A / w;"),
    ("conj_on_y1", "double p_im = a_im * b_re - a_re * b_im;", "double p_im = a_re * b_im - a_im * b_re;"),
    ("exponent_sign", "double e_re = cos(ang), e_im = sin(ang);", "double e_re = cos(ang), e_im = -sin(ang);"),
    ("lag_direction", "int64_t q = k + L + m;", "int64_t q = k - L + m;"),
    ("round_is_floor", "L = (int64_t)llround(D);", "L = (int64_t)floor(D);"),
    ("lagrange_weight", "w[0] = -mu * (mu - 1.0) * (mu - 2.0) / 6.0;", "w[0] = mu * (mu - 1.0) * (mu - 2.0) / 6.0;"),
    ("no_accumulation", "s += (acc_mode == 0) ? pw : sqrt(pw);", "s = (acc_mode == 0) ? pw : sqrt(pw);"),
    ("argmax_tie", "cost[p] > cost[best]", "cost[p] >= cost[best]"),
    ("zero_pad_edge", "if (q < 0 || q >= n) continue;", "if (q < 0 || q > n) continue;"),
    ("detect_tie_rule", "(v[q] == x && q < p)", "(v[q] == x && q > p)"),
    ("detect_window_short", "for (int64_t di = -r; di <= r && peak; ++di)", "for (int64_t di = -r; di < r && peak; ++di)"),
    ("detect_strict_threshold", "if (!(x >= threshold)) continue;", "if (!(x > threshold)) continue;"),
    ("detect_sort_order", "(v[tmp[b]] < v[key] ||", "(v[tmp[b]] > v[key] ||"),
    ("phase_not_reduced_wrong", "double ang = 2.0 * DGO_PI * (ph - floor(ph));", "double ang = DGO_PI * (ph - floor(ph));"),
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="dg_oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(workdir, name, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = os.path.join(workdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = oracle.build(force=True, src=path, out=os.path.join(workdir, f"lib{name}.so"))
    failed = []
    with oracle.using(so):
        for pin in oracle_pins.ALL_PINS:
            try:
                pin()
            except (AssertionError, ValueError):
                failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {name}"
