"""FP64 re-evaluation of near ties: the values that an FP32+compensated search re-evaluated
(FFE_FLAG_RESCORED) are FP64 k-sums, so they match the oracle to FP64 accuracy, far inside the
FP32 tolerance -- for the two-band model, each band alone, and the three-band model.

Each line's grid spans 0.01 around the oracle's coarse minimum (spacing 8e-5), so the points
around the minimum differ by less than the FP32 error bound and are re-evaluated; low T puts
most bands outside the exponentials' range (the compacted near-band path) and higher T puts
most inside it."""
import numpy as np
import pytest

import oracle
from oracle import search
from paper_1412_8754_gb300 import ffe

from test_gpu_parity import per_site

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11  # per site: FP64 sums of <= 4096 terms in another order


def windows(evaluate, k, hi=0.3, width=0.01):
    """Per line a window of the given width around the coarse (61-point) minimum of evaluate."""
    coarse = np.linspace(0.0, hi, 61)
    c = np.array([coarse[search.grid_argmin(evaluate(i, coarse))] for i in range(k)])
    lo = np.clip(c - width / 2, 0.0, None)
    return lo, lo + width


def lines(seed, k, T_range):
    rng = np.random.default_rng(seed)
    N = rng.choice(np.array([32, 48]), size=k).astype(np.int32)
    qx = rng.uniform(0.0, 0.3, k)
    h = rng.uniform(0.0, 0.08, k)
    T = rng.uniform(*T_range, k)
    return N, qx, h, T


@pytest.mark.parametrize("T_range", [(0.002, 0.004), (0.02, 0.05)])
def test_rescored_grid_minima_are_fp64(T_range):
    U, n = 4.0, 129
    N, qx, h, T = lines(51, 10, T_range)
    m = oracle.make_model(U=U)

    def ev(i, d):
        return oracle.omega_batch(m, int(N[i]), qx[i], 0.0, h[i], T[i], d)[0]

    lo, hi = windows(ev, len(N))
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        res = ctx.minimize(ffe.params(N, qx, 0.0, h, T, lo, hi, n))
    rescored = (res["flags"] & ffe.FFE_FLAG_RESCORED) != 0
    assert rescored.sum() >= 5, rescored
    for i in range(len(N)):
        ref = ev(i, np.linspace(lo[i], hi[i], n))
        assert res["idx_star"][i] == search.grid_argmin(ref), i
        if rescored[i]:
            assert per_site(res["omega_star"][i], ref[res["idx_star"][i]], N[i]) <= FP64_TOL, i


def test_rescored_band_minima_are_fp64():
    U, n = 4.0, 129
    N, qx, h, T = lines(52, 8, (0.002, 0.02))
    m = oracle.make_model(U=U)
    n_rescored = 0
    for b in range(2):
        def ev(i, d, b=b):
            return oracle.omega_batch(m, int(N[i]), qx[i], 0.0, h[i], T[i], d, bands=True)[1][:, b]

        lo, hi = windows(ev, len(N))
        with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
            res = ctx.minimize_bands(ffe.params(N, qx, 0.0, h, T, lo, hi, n))
        for i in range(len(N)):
            ref = ev(i, np.linspace(lo[i], hi[i], n))
            r = res[i, b]
            assert r["idx_star"] == search.grid_argmin(ref), (i, b)
            if r["flags"] & ffe.FFE_FLAG_RESCORED:
                n_rescored += 1
                assert per_site(r["omega_star"], ref[r["idx_star"]], N[i]) <= FP64_TOL, (i, b)
    assert n_rescored >= 4


def test_rescored_three_band_minima_are_fp64():
    from oracle import threeband

    N, U, n = 16, 1.2, 129
    rng = np.random.default_rng(53)
    k = 6
    qx = rng.uniform(0.0, 0.2, k)
    h = rng.uniform(0.0, 0.01, k)
    T = rng.uniform(0.0005, 0.003, k)

    def ev(i, d):
        return threeband.omega_batch(N, qx[i], 0.0, np.full(d.size, h[i]), np.full(d.size, T[i]), d, U=U)[0]

    lo, hi = windows(ev, k, hi=0.06, width=0.002)
    with ffe.Context(prec=ffe.FFE_FP32C, U=U, model="daghofer3") as ctx:
        res = ctx.minimize(ffe.params(N, qx, 0.0, h, T, lo, hi, n))
    rescored = (res["flags"] & ffe.FFE_FLAG_RESCORED) != 0
    assert rescored.any()
    for i in range(k):
        ref = ev(i, np.linspace(lo[i], hi[i], n))
        assert res["idx_star"][i] == search.grid_argmin(ref), i
        if rescored[i]:
            assert per_site(res["omega_star"][i], ref[res["idx_star"][i]], N) <= FP64_TOL * 0.08, i
