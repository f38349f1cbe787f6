"""The three-band model of App. B on the CUDA path vs its FP64 oracle, through the C ABI.

Energies are in eV; the per-site tolerances of the two-band tests (units of |t1|) are scaled
by |t1| = 0.08 eV: FP64 8e-11 eV, FP32+compensated 1.6e-8 eV.  Argmin indices and phase labels
must be identical to the oracle's."""
import numpy as np
import pytest

from oracle import search
from oracle import threeband as tb
from paper_1412_8754_gb300 import ffe

pytestmark = pytest.mark.gpu

T1 = 0.08
TOL = {ffe.FFE_FP64: 1e-9 * T1, ffe.FFE_FP32C: 2e-7 * T1}
PRECS = [ffe.FFE_FP64, ffe.FFE_FP32C]
U = 1.2


def ctx3(prec):
    return ffe.Context(prec=prec, U=U, model="daghofer3")


@pytest.mark.parametrize("prec", PRECS)
def test_omega_and_per_band_vs_oracle(prec):
    rng = np.random.default_rng(31)
    jobs = [(8, 0.0, 0.0), (16, 0.35, 0.0), (24, -0.2, 0.15), (16, 2.5, -1.1)]
    with ctx3(prec) as c:
        for N, qx, qy in jobs:
            n = 9
            h = rng.uniform(-0.04, 0.04, n)
            T = rng.uniform(0.0005, 0.01, n)
            d = rng.uniform(0.0, 0.05, n)
            ref, ref_b, _ = tb.omega_batch(N, qx, qy, h, T, d, U=U, bands=True)
            pts = ffe.points(N, qx, qy, h, T, d)
            got, got_b = c.omega(pts, bands=True)
            plain = c.omega(pts)
            assert got_b.shape == (n, 3)
            assert np.abs(plain - ref).max() / N**2 <= TOL[prec], (N, qx)
            assert np.abs(got - ref).max() / N**2 <= TOL[prec]
            assert np.abs(got_b - ref_b).max() / N**2 <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_grid_minimum_vs_oracle(prec):
    """BCS minimum of the three-band model (U = 1.2 eV: Delta* ~ 0.02 eV at N = 32)."""
    N, n = 32, 41
    grid = np.linspace(0.0, 0.05, n)
    cases = [(0.0, 0.0, 0.001), (0.0, 0.005, 0.002), (0.2, 0.0, 0.001), (0.0, 0.02, 0.001)]
    with ctx3(prec) as c:
        qx = np.array([q for q, _, _ in cases])
        h = np.array([x for _, x, _ in cases])
        T = np.array([t for _, _, t in cases])
        res, om, _ = c.minimize(ffe.params(N, qx, 0.0, h, T, 0.0, 0.05, n), want_grid=True)
    interior = 0
    for i, (q, hh, t) in enumerate(cases):
        ref, _, _ = tb.omega_batch(N, q, 0.0, hh, t, grid, U=U)
        assert np.abs(om[i * n:(i + 1) * n] - ref).max() / N**2 <= TOL[prec]
        j = search.grid_argmin(ref)
        interior += 0 < j < n - 1
        assert res["idx_star"][i] == j, (i, res["idx_star"][i], j)
    assert interior >= 1


@pytest.mark.parametrize("prec", PRECS)
def test_phase_scan_labels_vs_oracle(prec):
    N, n = 24, 21
    qx = np.array([0.0, 0.15, 0.3])
    h = np.array([0.0, 0.006, 0.02])
    T = np.array([0.001, 0.004])
    grid = np.linspace(0.0, 0.05, n)
    with ctx3(prec) as c:
        res, lab, best = c.phase_scan(N, qx, np.zeros(3), h, T, n=n, lo=0.0, hi=0.05)
        res2, lab2, best2 = c.phase_scan(N, qx, np.zeros(3), h, T, n=n, lo=0.0, hi=0.05)  # cached plan
    for name in res.dtype.names:  # one scan, executed twice: the same bits
        assert np.array_equal(res[name], res2[name], equal_nan=True), name
    assert np.array_equal(lab, lab2) and np.array_equal(best, best2)
    star = np.zeros((3, len(h) * len(T)))
    zero = np.zeros_like(star)
    for q in range(3):
        for ih in range(len(h)):
            for it in range(len(T)):
                ref, _, _ = tb.omega_batch(N, qx[q], 0.0, h[ih], T[it], grid, U=U)
                j = search.grid_argmin(ref)
                pt = ih * len(T) + it
                assert res["idx_star"][q, pt] == j
                star[q, pt], zero[q, pt] = ref[j], ref[0]
    for pt in range(star.shape[1]):
        want, wq = search.phase_label(star[:, pt], zero[:, pt], qx == 0.0)
        assert lab[pt] == want and best[pt] == wq, (pt, lab[pt], want)
    assert set(lab.tolist()) >= {0, 1}  # both normal and BCS points


def test_per_band_minimisation_three_bands():
    N, n = 24, 31
    grid = np.linspace(0.0, 0.05, n)
    h = np.array([0.0, 0.004])
    T = np.array([0.001, 0.002])
    with ctx3(ffe.FFE_FP64) as c:
        res = c.minimize_bands(ffe.params(N, 0.0, 0.0, h, T, 0.0, 0.05, n))
    assert res.shape == (2, 3)
    for i in range(2):
        _, ob, _ = tb.omega_batch(N, 0.0, 0.0, h[i], T[i], grid, U=U, bands=True)
        for b in range(3):
            assert res[i, b]["idx_star"] == search.grid_argmin(ob[:, b]), (i, b)
