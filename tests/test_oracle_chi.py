"""Pins of the pair-susceptibility oracle (App. C)."""
import math

import numpy as np
import pytest

import oracle
from oracle import chi
from oracle import threeband as tb

TWO_PI = 2 * math.pi


def eig2(kx, ky):
    """Two-band energies from numpy's eigen-solver of the App. A matrix (not the oracle's formula)."""
    p = oracle.RAGHU2
    cx, cy, sx, sy = math.cos(kx), math.cos(ky), math.sin(kx), math.sin(ky)
    t11 = -2 * (p["t1"] * cx + p["t2"] * cy) - 4 * p["t3"] * cx * cy
    t22 = -2 * (p["t2"] * cx + p["t1"] * cy) - 4 * p["t3"] * cx * cy
    t12 = -4 * p["t4"] * sx * sy
    return np.linalg.eigvalsh(np.array([[t11, t12], [t12, t22]]))


def zero_t_closed_form(bands, mu, N, qx, qy, h, eta_amp):
    """T -> 0: f(x) -> theta(-x), so each term is eta^2 [theta(E_u) + theta(E_d) - 1] / (E_u + E_d)."""
    nb = len(bands(0.1, 0.2))
    acc = np.zeros((nb, nb))
    for j in range(N):
        for i in range(N):
            kx, ky = TWO_PI * i / N, TWO_PI * j / N
            eu = bands(kx, ky) - mu - h
            ed = bands(-kx - qx, -ky - qy) - mu + h
            eta2 = (eta_amp * math.cos(-kx - qx) * math.cos(-ky - qy)) ** 2
            for a in range(nb):
                for b in range(nb):
                    s = eu[a] + ed[b]
                    acc[a, b] += eta2 * (float(eu[a] > 0) + float(ed[b] > 0) - 1.0) / s
    return acc / N**2


@pytest.mark.parametrize("qx,qy,h", [(0.0, 0.0, 0.0), (0.6, 0.2, 0.07)])
def test_two_band_zero_temperature(qx, qy, h):
    m = oracle.make_model()
    N = 12
    got = chi.chi(m, N, qx, qy, h, 1e-7, eta_amp=4.0)
    ref = zero_t_closed_form(eig2, m.mu, N, qx, qy, h, 4.0)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12)


def test_three_band_zero_temperature():
    N, qx, qy, h = 10, 0.4, -0.3, 0.012
    got = chi.chi("daghofer3", N, qx, qy, h, 1e-8, eta_amp=4.0)
    ref = zero_t_closed_form(lambda a, b: tb.band_energies(a, b), tb.DAGHOFER3["mu"], N, qx, qy, h, 4.0)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("model", ["raghu2", "daghofer3"])
def test_intraband_chi_is_the_curvature_of_omega(model):
    """Omega_e(Delta) = Omega_e(0) + N^2 Delta^2 (1/U - chi_ee) + O(Delta^4) for the same pair
    momenta and form factor: App. C's q is the free energy's Q = -q with eta at the relative
    momentum (eta_at="relative"); q = 4 pi / N keeps k + Q/2 on the lattice, so both sums run
    over the same points."""
    N, h = 16, 0.03
    q = 4 * math.pi / N
    if model == "raghu2":
        m = oracle.make_model(U=2.0, eta_amp=1.0)
        T, U = 0.02, 2.0
        c = chi.chi(m, N, q, 0.0, h, T, eta_amp=1.0, eta_at="relative")

        def om_b(d):
            return oracle.omega(m, N, -q, 0.0, h, T, d, bands=True)[1]
    else:
        T, U = 0.003, 1.2
        c = chi.chi("daghofer3", N, q, 0.0, h, T, eta_amp=1.0, eta_at="relative")

        def om_b(d):
            return tb.omega_batch(N, -q, 0.0, h, T, d, U=U, bands=True)[1][0]
    d = 1e-4 if model == "raghu2" else 2e-5
    curv = (om_b(d) - om_b(0.0)) / (N**2 * d * d)
    for e in range(len(curv)):
        assert abs((1.0 / U - curv[e]) - c[e, e]) <= 2e-5 * abs(c[e, e]) + 1e-6, (e, c[e, e], 1 / U - curv[e])
