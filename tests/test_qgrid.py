"""Full-Brillouin-zone Q scan: the wedge and the map back to the grid (host logic), and, on the
GPU, the wedge scan against the scan of every grid point."""
import math

import numpy as np
import pytest

from paper_1412_8754_gb300 import qgrid


@pytest.mark.parametrize("n", [2, 4, 8, 10])
def test_wedge_is_one_point_per_orbit(n):
    w = qgrid.wedge(n)
    assert tuple(w[0]) == (0, 0)
    assert len(w) == (n // 2 + 1) * (n // 2 + 2) // 2
    pos = qgrid.wedge_position(n)
    # every grid point maps into the wedge, and the images of a point under the group
    # (swap, both mirrors, the half period a -> a + n) map to the same wedge point
    for a in range(n):
        for b in range(n):
            p = pos[a, b]
            for (x, y) in [(b, a), (-a, b), (a, -b), (a + n, b), (b, -a), (-b, -a)]:
                assert pos[x % n, y % n] == p
    # and every wedge point is reached
    assert set(pos.ravel().tolist()) == set(range(len(w)))


def test_odd_grid_rejected():
    with pytest.raises(ValueError):
        qgrid.wedge(7)


@pytest.mark.gpu
def test_wedge_scan_equals_full_grid_scan():
    from paper_1412_8754_gb300 import ffe

    N, U, nq, n = 16, 4.0, 8, 41
    h = np.array([0.0, 0.06, 0.12])
    T = np.array([0.003, 0.02])
    A, B = np.meshgrid(np.arange(nq), np.arange(nq), indexing="ij")
    qx_all = 2 * math.pi * A.ravel() / nq
    qy_all = 2 * math.pi * B.ravel() / nq
    pos = qgrid.wedge_position(nq).ravel()
    with ffe.Context(prec=ffe.FFE_FP64, U=U) as ctx:
        full, flab, fbest = ctx.phase_scan(N, qx_all, qy_all, h, T, n=n)
        wres, wlab, wbq, wq = qgrid.fbz_phase_scan(ctx, N, nq, h, T, n=n)
    assert len(wq) == 15 and len(qx_all) == 64
    # every grid Q has the minimum of its wedge representative
    np.testing.assert_allclose(full["omega_star"], wres["omega_star"][pos], rtol=0, atol=1e-9 * N * N)
    np.testing.assert_array_equal(full["idx_star"], wres["idx_star"][pos])
    assert np.array_equal(flab, wlab)
    # the best Q of the full scan is a symmetry image of the wedge scan's
    ok = fbest >= 0
    assert np.array_equal(ok, ~np.isnan(wbq[:, 0]))
    assert np.all(pos[fbest[ok]] == np.array([np.argmin(np.abs(wq - b).sum(1)) for b in wbq[ok]]))
