"""Edge cases of the boundary against the oracle and against closed forms: the smallest and the
largest lattice, empty inputs, the longest Delta grid, a vanishing form factor, and temperatures
far below and far above the band scale.

Tolerances (per lattice site, units of |t1|): FP64 1e-9, FP32+compensated 2e-7; argmin indices
identical to the oracle's.
"""
import numpy as np
import pytest

import oracle
from oracle import search
from paper_1412_8754_gb300 import ffe

pytestmark = pytest.mark.gpu

TOL = {ffe.FFE_FP64: 1e-9, ffe.FFE_FP32C: 2e-7}
PRECS = [ffe.FFE_FP64, ffe.FFE_FP32C]
U = 2.5

# Four points of the largest lattice the boundary accepts (N = 8192: 67 108 864 k-points, the
# lattice index's 26 bits full), different Q, h, T and Delta; the oracle's values are computed
# once for both precisions.
BIG = dict(N=8192, qx=np.array([0.3, 0.0, 0.1, 0.05]), qy=np.array([0.0, 0.0, 0.02, 0.0]),
           h=np.array([0.05, 0.0, 0.1, -0.03]), T=np.array([0.002, 0.01, 0.005, 0.02]),
           delta=np.array([0.1, 0.0, 0.05, 0.15]))


@pytest.fixture(scope="module")
def big_reference():
    m = oracle.make_model(U=U)
    ref, _, _ = oracle.omega_batch(m, BIG["N"], BIG["qx"], BIG["qy"], BIG["h"], BIG["T"], BIG["delta"])
    return ref


def per_site(a, b, N):
    return np.abs(np.asarray(a) - np.asarray(b)) / float(N) ** 2


def test_empty_inputs_are_rejected_and_the_context_stays_usable():
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        with pytest.raises(ffe.FFEError) as e:
            ctx.omega(ffe.points(16, [], 0.0, 0.0, 0.01, 0.1))
        assert e.value.status == ffe.FFE_EINVAL
        with pytest.raises(ffe.FFEError) as e:
            ctx.minimize(ffe.params(16, [], 0.0, 0.0, 0.01, 0.0, 0.2, 8))
        assert e.value.status == ffe.FFE_EINVAL
        with pytest.raises(ffe.FFEError) as e:
            ctx.minimize(ffe.params(16, 0.0, 0.0, 0.0, 0.01, 0.0, 0.2, 0))  # a grid of no points
        assert e.value.status == ffe.FFE_EINVAL
        with pytest.raises(ffe.FFEError):
            ctx.phase_scan(16, [0.0, 0.1], [0.0, 0.0], [], [0.01], n=8)  # no h
        got = ctx.omega(ffe.points(16, 0.1, 0.0, 0.02, 0.01, 0.1))
        m = oracle.make_model(U=U)
        ref, _, _ = oracle.omega_batch(m, 16, 0.1, 0.0, 0.02, 0.01, 0.1)
        assert per_site(got, ref, 16).max() <= TOL[ffe.FFE_FP32C]


@pytest.mark.parametrize("prec", PRECS)
def test_largest_lattice_vs_oracle(prec, big_reference):
    with ffe.Context(prec=prec, U=U) as ctx:
        got = ctx.omega(ffe.points(BIG["N"], BIG["qx"], BIG["qy"], BIG["h"], BIG["T"], BIG["delta"]))
    err = per_site(got, big_reference, BIG["N"])
    assert err.max() <= TOL[prec], err


@pytest.mark.parametrize("prec", PRECS)
def test_smallest_lattice_vs_oracle(prec):
    """N = 2 (the four k-points 0 and pi on each axis): Omega and the grid argmin."""
    m = oracle.make_model(U=U)
    rng = np.random.default_rng(5)
    qx, h, T = rng.uniform(-1, 1, 40), rng.uniform(-0.2, 0.2, 40), rng.uniform(0.001, 0.2, 40)
    d = rng.uniform(0, 0.4, 40)
    ref, _, _ = oracle.omega_batch(m, 2, qx, 0.0, h, T, d)
    with ffe.Context(prec=prec, U=U) as ctx:
        got = ctx.omega(ffe.points(2, qx, 0.0, h, T, d))
        res = ctx.minimize(ffe.params(2, qx[:6], 0.0, h[:6], T[:6], 0.0, 0.4, 101))
    assert per_site(got, ref, 2).max() <= TOL[prec]
    for i in range(6):
        want, _, _, _ = search.minimize_grid(m, 2, qx[i], 0.0, h[i], T[i], 0.0, 0.4, 101)
        assert res["idx_star"][i] == want


@pytest.mark.parametrize("prec,n", [(ffe.FFE_FP64, 65536), (ffe.FFE_FP32C, 4096)])
def test_longest_grids_keep_the_oracle_argmin(prec, n):
    """Delta grids up to the boundary's limit of 65 536 points (a step of 3e-6 on [0, 0.2]) on
    an 8 x 8 lattice at an interior BCS minimum: the argmin index is the oracle's."""
    m = oracle.make_model(U=4.0)
    with ffe.Context(prec=prec, U=4.0) as ctx:
        res = ctx.minimize(ffe.params(8, [0.0, 0.4], 0.0, [0.0, 0.05], 0.01, 0.0, 0.2, n))
    for i, (qx, h) in enumerate([(0.0, 0.0), (0.4, 0.05)]):
        want, dstar, _, om = search.minimize_grid(m, 8, qx, 0.0, h, 0.01, 0.0, 0.2, n)
        assert res["idx_star"][i] == want, (i, res["idx_star"][i], want)
        assert res["delta_star"][i] == dstar
        assert abs(res["omega_star"][i] - om[want]) / 64.0 <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_vanishing_form_factor_leaves_the_pairing_term(prec):
    """eta = 0: the quasiparticle energies no longer depend on Delta (R = |s|), so
    Omega(Delta) - Omega(0) = N^2 Delta^2 (1/U_0 + 1/U_1) exactly (Eq. freeene with the pairing
    term read as +Delta^2/U per k-point and band), and the grid minimum is Delta = 0."""
    N, d = 32, np.linspace(0.0, 0.2, 33)
    with ffe.Context(prec=prec, U=U, eta_amp=0.0) as ctx:
        om = ctx.omega(ffe.points(N, 0.2, 0.0, 0.04, 0.005, d))
        res = ctx.minimize(ffe.params(N, 0.2, 0.0, 0.04, 0.005, 0.0, 0.2, 33))
    want = om[0] + N * N * d ** 2 * (2.0 / U)
    assert per_site(om, want, N).max() <= TOL[prec]
    assert res["idx_star"][0] == 0 and res["delta_star"][0] == 0.0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("T", [1e-6, 3.0])
def test_extreme_temperatures_vs_oracle(prec, T):
    """T far below every band splitting (every log factor 1: the T -> 0 ground state) and far
    above the band width (every band near the Fermi surface on the scale of T): the whole Omega
    grid of six (q, h) lines against the oracle.  The FP32C error bound the library returns with
    each grid value (2^-17 |V| + 2^-22 ln2 N^2 T, V the Delta-dependent part) grows with T; at
    T = 3 its temperature term alone is 5e-7 per site, above the 2e-7 that holds for the
    workloads' T <= 0.03, so each value is held to the larger of the two."""
    N, n = 48, 16
    m = oracle.make_model(U=U)
    rng = np.random.default_rng(17)
    qx, h = rng.uniform(-0.6, 0.6, 6), rng.uniform(-0.15, 0.15, 6)
    with ffe.Context(prec=prec, U=U) as ctx:
        res, grid, err = ctx.minimize(ffe.params(N, qx, 0.0, h, T, 0.0, 0.3, n), want_grid=True)
    d = search.delta_grid(0.0, 0.3, n)
    ref, _, _ = oracle.omega_batch(m, N, np.repeat(qx, n), 0.0, np.repeat(h, n), T, np.tile(d, 6))
    tol = np.maximum(TOL[prec] * N * N, err)
    assert np.all(np.abs(grid - ref) <= tol), float((np.abs(grid - ref) / tol).max())
    if prec == ffe.FFE_FP64:
        assert np.all(err == 0.0)
    for i in range(6):
        assert res["idx_star"][i] == search.grid_argmin(ref[i * n:(i + 1) * n])
