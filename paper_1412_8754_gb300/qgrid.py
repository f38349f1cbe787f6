"""Full-Brillouin-zone pair-momentum scan (Alg. 1 over every Q of an n x n grid).

Alg. 1 searches Q over the whole first Brillouin zone.  Omega is invariant
under the point group of the square lattice acting on Q -- k_x <-> k_y swaps
T11 and T22, k_x -> -k_x flips the sign of T12 (App. A), neither changes the
bands -- and, on an even lattice, under Q -> Q + 2 pi e_x (both spins shift by
the lattice vector pi e_x; eta^2 is unchanged).  So the n x n grid
Q = 2 pi (a, b) / n (n even) needs only the wedge 0 <= b <= a <= n/2: about
n^2/8 of its points.  Every Q of the grid has the Omega of its wedge
representative, so the phase labels of the full scan are those of the wedge
scan.  This module builds the wedge (host-side planning; the scan itself is
ffe_phase_scan) and maps results back to the full grid.
"""
from __future__ import annotations

import math

import numpy as np

from . import ffe


def wedge(n: int):
    """Index pairs (a, b), 0 <= b <= a <= n/2, of the irreducible wedge of the n x n Q grid,
    Q = 2 pi (a, b) / n; (0, 0) first."""
    if n < 2 or n % 2:
        raise ValueError("the Q grid needs an even n >= 2")
    ab = [(a, b) for a in range(n // 2 + 1) for b in range(a + 1)]
    return np.array(ab, dtype=np.int64)


def representative(n: int, a, b):
    """Wedge index pair of grid point (a, b) (any integers): fold to [0, n), mirror to
    [0, n/2], order so that b <= a."""
    a = np.mod(np.asarray(a), n)
    b = np.mod(np.asarray(b), n)
    a = np.minimum(a, n - a)
    b = np.minimum(b, n - b)
    return np.maximum(a, b), np.minimum(a, b)


def wedge_position(n: int):
    """Array [n, n]: the position in wedge(n) of every grid point (a, b)."""
    w = wedge(n)
    pos = {(int(a), int(b)): i for i, (a, b) in enumerate(w)}
    A, B = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ra, rb = representative(n, A, B)
    return np.vectorize(lambda x, y: pos[(int(x), int(y))])(ra, rb)


def fbz_phase_scan(ctx: "ffe.Context", N: int, n_q: int, h, T, search=ffe.FFE_SEARCH_GRID, n=256, lo=0.0,
                   hi=0.2, stream=None):
    """Phase scan with Q over the whole n_q x n_q grid of the Brillouin zone (N even).

    Returns (per_line[n_wedge, n_pts], labels[n_pts], best_q[n_pts, 2], wedge_q[n_wedge, 2]):
    per-line results and labels of the wedge scan, the best Q of each point as (qx, qy) of
    its wedge representative (NaN where the label is normal), and the wedge's Q values."""
    if N % 2:
        raise ValueError("the half-period reduction needs an even lattice")
    w = wedge(n_q)
    q = 2.0 * math.pi * w / n_q
    res, labels, best = ctx.phase_scan(N, q[:, 0], q[:, 1], h, T, search=search, n=n, lo=lo, hi=hi,
                                       stream=stream)
    bq = np.full((len(labels), 2), np.nan)
    ok = best >= 0
    bq[ok] = q[best[ok]]
    return res, labels, bq, q
