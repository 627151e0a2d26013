"""Pins of the oracle's parabolic sub-node estimate (oracle.subcell): exact on
a sampled concave quadratic, zero at edges, on flat or convex triples and
next to non-finite values, and never beyond half a node."""
import math

import numpy as np
import pytest

import oracle


def test_exact_on_a_sampled_quadratic():
    i0, j0 = 5.3, 7.8
    ii, jj = np.mgrid[0:12, 0:15]
    f = 100.0 - 2.5 * (ii - i0) ** 2 - 0.7 * (jj - j0) ** 2
    i, j = np.unravel_index(np.argmax(f), f.shape)
    assert (i, j) == (5, 8)
    di, dj = oracle.subcell(f, i, j)
    assert di == pytest.approx(0.3, abs=1e-12) and dj == pytest.approx(-0.2, abs=1e-12)


def test_edges_flat_convex_and_nan():
    f = np.array([[3.0, 1.0, 0.0], [2.0, 0.5, 0.0], [1.0, 0.2, 0.0]])
    assert oracle.subcell(f, 0, 0) == (0.0, 0.0)          # corner: no neighbours on one side
    flat = np.ones((3, 3))
    assert oracle.subcell(flat, 1, 1) == (0.0, 0.0)       # a - 2b + d = 0
    convex = np.array([[0, 5, 0], [5, 1, 5], [0, 5, 0]], dtype=float)
    assert oracle.subcell(convex, 1, 1) == (0.0, 0.0)     # a - 2b + d > 0
    g = np.array([[0, 1, 0], [np.nan, 3, 1], [0, 1, 0]], dtype=float)
    di, dj = oracle.subcell(g, 1, 1)
    assert dj == 0.0 and di == 0.0                        # nan neighbour in the row; column flat-symmetric


def test_offset_stays_within_half_a_node():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        b = rng.uniform(0, 1)
        a, d = b - rng.uniform(0, 1), b - rng.uniform(0, 1)  # b is the maximum of the triple
        x = oracle.parabola_offset(a, b, d)
        assert -0.5 <= x <= 0.5
        if a < b and d < b:
            # the parabola's vertex value is at least b
            den = a - 2 * b + d
            y = b - 0.125 * (a - d) ** 2 / den
            assert y >= b - 1e-12
    assert oracle.parabola_offset(0.0, 1.0, 0.0) == 0.0
    assert oracle.parabola_offset(1.0, 1.0, 0.0) == pytest.approx(-0.5)  # equal at -1 and 0: vertex at -0.5
    assert oracle.parabola_offset(0.0, 1.0, 1.0) == pytest.approx(0.5)
