"""Coarse delay-Doppler maps back-projected onto a footprint grid, FP64.

TEST INFRASTRUCTURE: only ``tests/`` may import this module. It is the CPU
oracle for the device's coarse maps (the input of the learned proposal) and
shares no code with them; the per-node geometry comes from the C oracle
(Eq. 3-10, ``dgo_node_geometry``).

Definitions, per snapshot k with captures y1, y2 of N samples (samples outside
[0, N) are zero):

* The cross-ambiguity function (the delay-Doppler map of the classical
  two-step TDOA/FDOA method the paper contrasts with, Sec. I) at integer lag l
  and FDOA nu is the correlation of Eq. 11 before the magnitude:
      X(l, nu) = sum_n y1[n] conj(y2[n + l]) exp(j 2 pi nu n).
* It is sampled at the lags l0 .. l0 + nlag - 1 spanned by the grid nodes'
  lags round(D) (Eq. 9, half away from zero) and at Q bin frequencies
  nu_q = nu_lo + q delta, delta = (nu_hi - nu_lo) / (Q - 1), where
  [nu_lo, nu_hi] is the nodes' FDOA range (Eq. 10).
* It is evaluated in chunks of M samples: the lag product of each chunk is
  turned at the centre frequency nu_c = (nu_lo + nu_hi) / 2 and summed,
      P_b(l) = sum_{m < M} y1[bM + m] conj(y2[bM + m + l]) exp(j 2 pi nu_c (bM + m)),
  and the chunks are combined at each bin,
      Xc(l, q) = sum_b exp(j 2 pi (nu_q - nu_c) b M) P_b(l).
  Xc = X(l, nu_q) when M = 1 or nu_q = nu_c; otherwise sample n = bM + m is
  turned by nu_q n - (nu_q - nu_c) m instead of nu_q n, so
      |Xc - X| <= 2 pi |nu_q - nu_c| (M - 1) sum_n |y1[n]| |y2[n + l]|.
* A(l, q) = |Xc(l, q)|^2 and mu = the mean of A over its nlag x Q entries.
* Cell (i, j) of the footprint is the quadrilateral of nodes (i, j),
  (i + 1, j), (i, j + 1), (i + 1, j + 1). Its coarse value is the largest A / mu
  over the lags from the smallest to the largest of its corners' lags, and the
  bins from floor((nu_min - nu_lo) / delta) to ceil((nu_max - nu_lo) / delta)
  (clipped to [0, Q - 1]; every bin when delta = 0), nu_min and nu_max being
  its corners' extreme FDOAs: a max-pool of the map over the delay-Doppler box
  the cell covers. When mu = 0 (captures of zeros) every coarse value is 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import iq_to_f64, node_geometry


def round_half_away(D):
    """Eq. 9's rounding, half away from zero, exactly."""
    D = np.asarray(D, dtype=np.float64)
    a = np.abs(D)
    f = np.floor(a)
    up = (a - f) >= 0.5
    return (np.sign(D) * (f + up)).astype(np.int64)


def step_params(lag_k, nu_k, Q):
    """(l0, nlag, nu_lo, delta, nu_c) of one snapshot from its node lags and
    FDOAs."""
    l0, l1 = int(lag_k.min()), int(lag_k.max())
    lo, hi = float(nu_k.min()), float(nu_k.max())
    delta = (hi - lo) / (Q - 1) if Q > 1 else 0.0
    return l0, l1 - l0 + 1, lo, delta, 0.5 * (lo + hi)


def caf(y1, y2, l0, nlag, nu_lo, delta, nu_c, Q, M):
    """A(l, q) = |Xc(l0 + l, nu_lo + q delta)|^2, shape (nlag, Q); y1, y2 are
    complex (N,)."""
    N = y1.size
    nb = -(-N // M)
    n = np.arange(N)
    turn = np.exp(2j * math.pi * nu_c * n)
    nu_q = nu_lo + np.arange(Q) * delta
    b = np.arange(nb)
    comb = np.exp(2j * math.pi * np.outer(nu_q - nu_c, b * M))   # (Q, nb)
    A = np.empty((nlag, Q))
    for t in range(nlag):
        l = l0 + t
        y2s = np.zeros(N, dtype=np.complex128)
        lo, hi = max(0, -l), min(N, N - l)
        if hi > lo:
            y2s[lo:hi] = y2[lo + l:hi + l]
        r = np.zeros(nb * M, dtype=np.complex128)
        r[:N] = y1 * np.conj(y2s) * turn
        P = r.reshape(nb, M).sum(axis=1)
        A[t] = np.abs(comb @ P) ** 2
    return A


def backproject(A, mu, lag_k, nu_k, l0, nu_lo, delta):
    """Coarse value of every cell, shape (nlat - 1, nlon - 1)."""
    nlag, Q = A.shape
    nlat, nlon = lag_k.shape
    out = np.empty((nlat - 1, nlon - 1))
    for i in range(nlat - 1):
        for j in range(nlon - 1):
            L = lag_k[i:i + 2, j:j + 2]
            V = nu_k[i:i + 2, j:j + 2]
            la, lb = int(L.min()) - l0, int(L.max()) - l0
            if delta > 0.0:
                qa = max(0, int(math.floor((V.min() - nu_lo) / delta)))
                qb = min(Q - 1, int(math.ceil((V.max() - nu_lo) / delta)))
            else:
                qa, qb = 0, Q - 1
            out[i, j] = A[la:lb + 1, qa:qb + 1].max() / mu if mu > 0.0 else 0.0
    return out


def coarse_maps(grid, ephem, fs, fc, y1, y2, Q, M, want_caf=False):
    """Coarse maps (K, nlat - 1, nlon - 1) of a scene; with want_caf also the
    per-snapshot (params, A, mu). y1, y2: (K, N, 2) in any storage type."""
    D, nu = node_geometry(grid, ephem, fs, fc)
    lag = round_half_away(D)
    a, b = iq_to_f64(y1), iq_to_f64(y2)
    K = a.shape[0]
    maps, extra = [], []
    for k in range(K):
        l0, nlag, lo, delta, nc = step_params(lag[k], nu[k], Q)
        A = caf(a[k, :, 0] + 1j * a[k, :, 1], b[k, :, 0] + 1j * b[k, :, 1], l0, nlag, lo, delta, nc, Q, M)
        mu = float(A.mean())
        maps.append(backproject(A, mu, lag[k], nu[k], l0, lo, delta))
        extra.append(((l0, nlag, lo, delta, nc), A, mu))
    maps = np.stack(maps)
    return (maps, extra) if want_caf else maps
