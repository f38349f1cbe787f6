"""Pins of the three-band oracle (App. B): none of them re-calls the eigen-solver it uses."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import threeband as tb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "daghofer3_app_b.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if len(line) == 2:
            vals[line[0]] = float(line[1])
    return vals


def test_parameters_are_the_printed_ones():
    g = golden()
    for k, v in tb.DAGHOFER3.items():
        assert g[k] == v, k


def test_printed_filling():
    """App. B: n = 4 particles per site at mu = 0.4748 eV (two spins, three bands, T = 0)."""
    g = golden()
    assert abs(tb.filling(256, g["mu"]) - g["n"]) < 2e-3
    assert tb.filling(128, g["mu"] - 0.03) < g["n"] < tb.filling(128, g["mu"] + 0.03)


def det3(T):
    """Determinant of a 3x3 matrix by the rule of Sarrus, written out."""
    return (T[0, 0] * T[1, 1] * T[2, 2] + T[0, 1] * T[1, 2] * T[2, 0] + T[0, 2] * T[1, 0] * T[2, 1]
            - T[0, 2] * T[1, 1] * T[2, 0] - T[0, 0] * T[1, 2] * T[2, 1] - T[0, 1] * T[1, 0] * T[2, 2])


def test_eigenvalues_satisfy_trace_determinant_and_minors():
    rng = np.random.default_rng(3)
    for kx, ky in rng.uniform(-math.pi, math.pi, (50, 2)):
        T = tb.hopping_matrix(kx, ky)
        e = tb.band_energies(kx, ky)
        assert np.all(np.diff(e) >= 0)
        assert abs(e.sum() - (T[0, 0] + T[1, 1] + T[2, 2]).real) < 1e-13
        assert abs(np.prod(e) - det3(T).real) < 1e-13
        minors = (T[0, 0] * T[1, 1] - T[0, 1] * T[1, 0] + T[0, 0] * T[2, 2] - T[0, 2] * T[2, 0]
                  + T[1, 1] * T[2, 2] - T[1, 2] * T[2, 1]).real
        assert abs(e[0] * e[1] + e[0] * e[2] + e[1] * e[2] - minors) < 1e-13
        assert np.allclose(T, np.conj(T.T))


def test_lattice_symmetries_of_the_bands():
    """kx <-> ky swaps T11/T22 and T13/T23; kx -> -kx conjugates the off-diagonals."""
    rng = np.random.default_rng(4)
    k = rng.uniform(-math.pi, math.pi, (40, 2))
    e = tb.band_energies(k[:, 0], k[:, 1])
    np.testing.assert_allclose(tb.band_energies(k[:, 1], k[:, 0]), e, atol=1e-13)
    np.testing.assert_allclose(tb.band_energies(-k[:, 0], k[:, 1]), e, atol=1e-13)
    np.testing.assert_allclose(tb.band_energies(k[:, 0] + 2 * math.pi, k[:, 1]), e, atol=1e-13)


@pytest.mark.parametrize("qx,h,T", [(0.0, 0.0, 0.002), (0.3, 0.02, 0.001)])
def test_delta_zero_is_free_fermions_per_band(qx, h, T):
    """At Delta = 0 each band gives -T sum_{k,sigma} ln(1 + exp(-E/T)) at k + Q/2."""
    N = 16
    mu = tb.DAGHOFER3["mu"]
    e_up, _ = tb.band_grids(N, qx, 0.0)
    _, ob, _ = tb.omega_batch(N, qx, 0.0, h, T, 0.0, U=1.2, bands=True)
    for b in range(3):
        terms = [-T * np.logaddexp(0.0, -(e_up[..., b] - mu - s * h) / T) for s in (+1, -1)]
        ref = math.fsum(np.concatenate([t.ravel() for t in terms]))
        assert abs(ob[0, b] - ref) <= 1e-12 * abs(ref), b


def test_zero_temperature_limit_is_ground_state():
    """T -> 0: each (band, k) pair contributes its lowest many-body level plus Delta^2/U."""
    N, qx, h, delta, U, T = 8, 0.4, 0.01, 0.02, 1.2, 1e-10
    mu = tb.DAGHOFER3["mu"]
    e_up, e_dn = tb.band_grids(N, qx, 0.0)
    k = 2 * math.pi * np.arange(N) / N
    terms = []
    for j in range(N):
        for i in range(N):
            gap = delta * math.cos(k[i]) * math.cos(k[j])
            for b in range(3):
                eu, ed = e_up[j, i, b] - mu - h, e_dn[j, i, b] - mu + h
                levels = [0.0, eu, ed, 0.5 * (eu + ed) - math.hypot(0.5 * (eu + ed), gap)]
                terms.append(min(levels) + delta * delta / U)
    om, _, _ = tb.omega_batch(N, qx, 0.0, h, T, delta, U=U)
    assert abs(om[0] - math.fsum(terms)) < 1e-9


def test_given_energies_path_matches_the_two_band_closed_form():
    """The nb-band k-sum fed with the two-band energies reproduces the two-band oracle, each band
    with its own coupling."""
    m = oracle.make_model(U=2.0, U_band=(1.5, 3.0))
    N, qx, qy, h, T, d = 12, 0.35, 0.1, 0.05, 0.01, 0.12
    e_up = np.ascontiguousarray(oracle.band_grid(m, N, qx, qy))
    k = 2 * math.pi * np.arange(N) / N
    e_dn = np.zeros_like(e_up)
    for j in range(N):
        for i in range(N):
            e_dn[j, i] = oracle.band_energies(m, -k[i] + qx / 2, -k[j] + qy / 2)
    out = np.zeros(1)
    ob = np.zeros(2)
    L = oracle.lib()
    Ub = np.array([1.5, 3.0])
    L.ffeo_omega_given(2, N, oracle._dp(e_up), oracle._dp(e_dn), 1.0, m.mu, oracle._dp(Ub), h, T, d,
                       oracle._dp(out), oracle._dp(ob))
    ref, rb = oracle.omega(m, N, qx, qy, h, T, d, bands=True)
    assert abs(out[0] - ref) <= 1e-12 * abs(ref)
    np.testing.assert_allclose(ob, rb, rtol=1e-12)
