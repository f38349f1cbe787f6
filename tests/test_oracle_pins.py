"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula for Omega: each compares it with
an independent route (a library eigen-solver, a many-body trace, a closed form,
a symmetry, a stationarity condition, a number the paper prints).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import search

RNG = np.random.default_rng(20141231)
TWO_PI = 2.0 * math.pi


def hopping_matrix(p, kx, ky):
    """App. A: the 2x2 orbital hopping matrix T_k (d_xz, d_yz)."""
    cx, cy, sx, sy = math.cos(kx), math.cos(ky), math.sin(kx), math.sin(ky)
    t11 = -2 * (p["t1"] * cx + p["t2"] * cy) - 4 * p["t3"] * cx * cy
    t22 = -2 * (p["t2"] * cx + p["t1"] * cy) - 4 * p["t3"] * cx * cy
    t12 = -4 * p["t4"] * sx * sy
    return np.array([[t11, t12], [t12, t22]])


def bands_eigvalsh(p, kx, ky):
    return np.linalg.eigvalsh(hopping_matrix(p, kx, ky))  # ascending: [E_-, E_+]


def pair_free_energy_fock(e_up, e_dn, gap, T):
    """-T ln Tr exp(-H/T) for one (k up, -k+q down) pair of modes.

    H = E_up n_up + E_dn n_dn + gap (d_up d_dn + h.c.) on the 4-state Fock space
    |0>, |up>, |dn>, |up dn>; the pairing term couples |0> and |up dn> with a
    fermion sign of -1.  This is the many-body partition function, with no use
    of the Bogoliubov formula."""
    H = np.zeros((4, 4))
    H[1, 1] = e_up
    H[2, 2] = e_dn
    H[3, 3] = e_up + e_dn
    H[0, 3] = H[3, 0] = -gap
    lam = np.linalg.eigvalsh(H)
    x = -lam / T
    xm = x.max()
    return -T * (xm + math.log(np.exp(x - xm).sum()))


def omega_bruteforce(p, U, eta_amp, N, qx, qy, h, T, delta):
    """Whole-lattice Omega from per-pair many-body traces (no Eq. enequasiparticle)."""
    terms = []
    for j in range(N):
        for i in range(N):
            kx, ky = TWO_PI * i / N, TWO_PI * j / N
            e_kq = bands_eigvalsh(p, kx + qx / 2, ky + qy / 2)
            e_mkq = bands_eigvalsh(p, -kx + qx / 2, -ky + qy / 2)
            gap = delta * eta_amp * math.cos(kx) * math.cos(ky)
            for b in range(2):
                e_up = e_kq[b] - p["mu"] - h
                e_dn = e_mkq[b] - p["mu"] + h
                terms.append(pair_free_energy_fock(e_up, e_dn, gap, T))
                terms.append(delta * delta / U)
    return math.fsum(terms)


# ---------------------------------------------------------------- App. A bands
def test_band_energies_match_library_eigensolver():
    m = oracle.make_model()
    for kx, ky in RNG.uniform(-2 * math.pi, 2 * math.pi, size=(200, 2)):
        e = oracle.band_energies(m, kx, ky)
        ref = bands_eigvalsh(oracle.RAGHU2, kx, ky)
        np.testing.assert_allclose(e, ref, rtol=0, atol=1e-13)


def test_half_filling_at_paper_mu():
    """App. A: mu = 1.54 |t1| gives two electrons per site (two bands, two spins).

    The paper prints mu to two decimals; with dn/dmu ~ 0.75 that fixes n to
    within ~0.004 of 2, and n(1.50) < 2 < n(1.58) brackets the rounding."""
    m = oracle.make_model()
    N = 256
    E = oracle.band_grid(m, N)

    def density(mu):
        return 2.0 * np.count_nonzero(E < mu) / N**2

    assert abs(density(1.54) - 2.0) < 0.005
    assert density(1.50) < 2.0 < density(1.58)


def test_band_energies_even_in_k():
    """Sec. 3 (BCS simplification): E_{eps,-k} = E_{eps,k}."""
    m = oracle.make_model()
    for kx, ky in RNG.uniform(-math.pi, math.pi, size=(50, 2)):
        np.testing.assert_allclose(oracle.band_energies(m, kx, ky),
                                   oracle.band_energies(m, -kx, -ky), rtol=0, atol=1e-14)


# ---------------------------------------------------- Eq. enequasiparticle / F
def test_quasiparticle_vieta_identities():
    for e_up, e_dn, gap in RNG.normal(0, 2, size=(200, 3)):
        ep, em = oracle.quasiparticle(e_up, e_dn, gap)
        assert ep >= em
        assert abs((ep + em) - (e_up - e_dn)) < 1e-13
        assert abs(ep * em - (-e_up * e_dn - gap * gap)) < 1e-12


def test_F_matches_logaddexp():
    for E, T in zip(RNG.normal(0, 3, 300), 10 ** RNG.uniform(-5, 0, 300)):
        ref = -T * np.logaddexp(0.0, -E / T)
        assert abs(oracle.F(E, T) - ref) <= 1e-14 * max(1.0, abs(ref))


def test_pair_term_equals_many_body_trace():
    """F(E+) + F(E-) + E_dn is the exact grand potential of one pair (Eq. freeene)."""
    for _ in range(300):
        e_up, e_dn = RNG.normal(0, 2, 2)
        gap = RNG.normal(0, 0.3)
        T = 10 ** RNG.uniform(-4, -0.5)
        ep, em = oracle.quasiparticle(e_up, e_dn, gap)
        lhs = oracle.F(ep, T) + oracle.F(em, T) + e_dn
        rhs = pair_free_energy_fock(e_up, e_dn, gap, T)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


# ------------------------------------------------------------- whole lattice
@pytest.mark.parametrize("qx,qy,h,T,delta,U,eta", [
    (0.0, 0.0, 0.0, 0.005, 0.0, 2.0, 1.0),
    (0.0, 0.0, 0.0, 0.005, 0.12, 4.0, 1.0),
    (0.31, 0.0, 0.07, 0.002, 0.08, 2.0, 1.0),
    (0.2, -0.45, 0.11, 0.03, 0.19, 2.0, 4.0),
    (1.7, 0.4, -0.05, 1e-4, 0.05, 3.0, 1.0),
])
def test_bruteforce_8x8_many_body(qx, qy, h, T, delta, U, eta):
    m = oracle.make_model(U=U, eta_amp=eta)
    got = oracle.omega(m, 8, qx, qy, h, T, delta)
    ref = omega_bruteforce(oracle.RAGHU2, U, eta, 8, qx, qy, h, T, delta)
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_bands_sum_to_total():
    m = oracle.make_model()
    tot, ob = oracle.omega(m, 16, 0.4, 0.0, 0.06, 0.01, 0.1, bands=True)
    assert abs(ob.sum() - tot) <= 1e-12 * abs(tot)


@pytest.mark.parametrize("qx,qy,h,T", [(0.0, 0.0, 0.0, 0.005), (0.37, 0.0, 0.08, 0.002),
                                       (0.5, 0.9, -0.03, 0.02)])
def test_delta_zero_is_free_fermions(qx, qy, h, T):
    """At Delta = 0 Omega = -T sum_{k,eps,sigma} ln(1 + exp(-E_{eps sigma}(k+Q/2)/T)).

    Both spins are evaluated at k + Q/2 here: the oracle's spin-down momenta
    -k + Q/2 are a permutation of the same lattice, so this is an independent
    route through the lattice sum."""
    m = oracle.make_model()
    N = 32
    ks = TWO_PI * np.arange(N) / N
    terms = []
    for ky in ks:
        for kx in ks:
            e = bands_eigvalsh(oracle.RAGHU2, kx + qx / 2, ky + qy / 2)
            for sigma in (+1, -1):
                x = e - oracle.RAGHU2["mu"] - sigma * h
                terms.extend(-T * np.logaddexp(0.0, -x / T))
    ref = math.fsum(terms)
    got = oracle.omega(m, N, qx, qy, h, T, 0.0)
    assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("qx,h,T", [(0.0, 0.0, 0.005), (0.37, 0.08, 0.002)])
def test_per_band_delta_zero_is_free_fermions(qx, h, T):
    """Per band eps at Delta = 0: Omega_eps = -T sum_{k,sigma} ln(1 + exp(-E_{eps sigma}/T)),
    with the bands ordered lower (0), upper (1) as the eigenvalues of the App. A matrix."""
    m = oracle.make_model()
    N = 24
    ks = TWO_PI * np.arange(N) / N
    terms = [[], []]
    for ky in ks:
        for kx in ks:
            e = bands_eigvalsh(oracle.RAGHU2, kx + qx / 2, ky)
            for b in range(2):
                for sigma in (+1, -1):
                    x = e[b] - oracle.RAGHU2["mu"] - sigma * h
                    terms[b].append(-T * np.logaddexp(0.0, -x / T))
    _, ob = oracle.omega(m, N, qx, 0.0, h, T, 0.0, bands=True)
    for b in range(2):
        ref = math.fsum(terms[b])
        assert abs(ob[b] - ref) <= 1e-12 * abs(ref), (b, ob[b], ref)


def test_per_band_zero_temperature_limit():
    """T -> 0 per band: each pair of band eps contributes its lowest many-body level plus
    Delta^2 / U."""
    m = oracle.make_model(U=2.0)
    N, qx, h, delta, T = 8, 0.4, 0.05, 0.1, 1e-9
    ks = TWO_PI * np.arange(N) / N
    terms = [[], []]
    for ky in ks:
        for kx in ks:
            e_kq = bands_eigvalsh(oracle.RAGHU2, kx + qx / 2, ky)
            e_mkq = bands_eigvalsh(oracle.RAGHU2, -kx + qx / 2, -ky)
            gap = delta * math.cos(kx) * math.cos(ky)
            for b in range(2):
                eu, ed = e_kq[b] - 1.54 - h, e_mkq[b] - 1.54 + h
                levels = [0.0, eu, ed, 0.5 * (eu + ed) - math.hypot(0.5 * (eu + ed), gap)]
                terms[b].append(min(levels) + delta * delta / 2.0)
    _, ob = oracle.omega(m, N, qx, 0.0, h, T, delta, bands=True)
    for b in range(2):
        assert abs(ob[b] - math.fsum(terms[b])) < 1e-9, b


def test_q_point_group_and_half_period():
    """The full-FBZ q scan rests on these: the model is symmetric under k_x <-> k_y and
    k_x -> -k_x (App. A: T11 <-> T22, T12 -> -T12 leave the bands unchanged), so
    Omega(qx, qy) = Omega(qy, qx) = Omega(-qx, qy); on an even lattice Q -> Q + 2 pi e_x shifts
    both spins by the lattice vector pi e_x and eta^2 is unchanged."""
    m = oracle.make_model(U=2.0)
    N = 20
    for qx, qy, h, T, d in [(0.7, 0.25, 0.05, 0.004, 0.11), (2.1, -1.3, 0.1, 0.02, 0.05)]:
        ref = oracle.omega(m, N, qx, qy, h, T, d)
        tol = 1e-12 * abs(ref)
        assert abs(oracle.omega(m, N, qy, qx, h, T, d) - ref) <= tol
        assert abs(oracle.omega(m, N, -qx, qy, h, T, d) - ref) <= tol
        assert abs(oracle.omega(m, N, qx, -qy, h, T, d) - ref) <= tol
        assert abs(oracle.omega(m, N, qx + 2 * math.pi, qy, h, T, d) - ref) <= tol
        assert abs(oracle.omega(m, N, qx, qy - 2 * math.pi, h, T, d) - ref) <= tol
    # an odd lattice has no pi shift: the half period does not hold there
    a = oracle.omega(m, 9, 0.7, 0.25, 0.05, 0.004, 0.11)
    b = oracle.omega(m, 9, 0.7 + 2 * math.pi, 0.25, 0.05, 0.004, 0.11)
    assert abs(a - b) > 1e-9 * abs(a)


def test_zero_temperature_limit_is_ground_state():
    """T -> 0: each pair contributes its lowest many-body level."""
    m = oracle.make_model(U=2.0)
    N, qx, h, delta, T = 8, 0.4, 0.05, 0.1, 1e-9
    ks = TWO_PI * np.arange(N) / N
    terms = []
    for ky in ks:
        for kx in ks:
            e_kq = bands_eigvalsh(oracle.RAGHU2, kx + qx / 2, ky)
            e_mkq = bands_eigvalsh(oracle.RAGHU2, -kx + qx / 2, -ky)
            gap = delta * math.cos(kx) * math.cos(ky)
            for b in range(2):
                eu, ed = e_kq[b] - 1.54 - h, e_mkq[b] - 1.54 + h
                levels = [0.0, eu, ed, 0.5 * (eu + ed) - math.hypot(0.5 * (eu + ed), gap)]
                terms.append(min(levels) + delta * delta / 2.0)
    assert abs(oracle.omega(m, N, qx, 0.0, h, T, delta) - math.fsum(terms)) < 1e-9


def test_symmetries():
    m = oracle.make_model(U=2.0)
    N = 24
    for qx, qy, h, T, d in [(0.3, 0.0, 0.07, 0.004, 0.09), (0.5, 0.2, 0.1, 0.02, 0.15)]:
        ref = oracle.omega(m, N, qx, qy, h, T, d)
        tol = 1e-13 * abs(ref)
        assert abs(oracle.omega(m, N, -qx, -qy, h, T, d) - ref) <= tol   # Q -> -Q
        assert abs(oracle.omega(m, N, qx, qy, -h, T, d) - ref) <= tol    # h -> -h
        assert abs(oracle.omega(m, N, qx, qy, h, T, -d) - ref) <= tol    # Delta -> -Delta
        assert abs(oracle.omega(m, N, qx + 4 * math.pi, qy, h, T, d) - ref) <= 1e-12 * abs(ref)


def test_lattice_vector_shift_at_delta_zero():
    """q/2 a lattice vector only relabels k, so the normal state is unchanged."""
    m = oracle.make_model()
    N = 32
    ref = oracle.omega(m, N, 0.0, 0.0, 0.06, 0.01, 0.0)
    for mshift in (1, 3, 7):
        got = oracle.omega(m, N, 4 * math.pi * mshift / N, 0.0, 0.06, 0.01, 0.0)
        assert abs(got - ref) <= 1e-13 * abs(ref)


def _analytic_dOmega(p, U, N, qx, qy, h, T, delta):
    """dOmega/dDelta = sum_k,eps [f(E+) - f(E-)] Delta eta^2 / R + 4 N^2 Delta / U,
    f the Fermi function (derivative of F), R the square root in Eq. enequasiparticle."""
    ks = TWO_PI * np.arange(N) / N
    acc = []
    for ky in ks:
        for kx in ks:
            e_kq = bands_eigvalsh(p, kx + qx / 2, ky + qy / 2)
            e_mkq = bands_eigvalsh(p, -kx + qx / 2, -ky + qy / 2)
            eta = math.cos(kx) * math.cos(ky)
            for b in range(2):
                eu, ed = e_kq[b] - p["mu"] - h, e_mkq[b] - p["mu"] + h
                dd, s = 0.5 * (eu - ed), 0.5 * (eu + ed)
                R = math.sqrt(s * s + (delta * eta) ** 2)
                fp = 0.5 * (1 - math.tanh((dd + R) / (2 * T)))
                fm = 0.5 * (1 - math.tanh((dd - R) / (2 * T)))
                acc.append((fp - fm) * delta * eta * eta / R)
    return math.fsum(acc) + 4 * N * N * delta / U


@pytest.mark.parametrize("qx,h,T,delta", [(0.0, 0.0, 0.01, 0.1), (0.35, 0.06, 0.02, 0.07)])
def test_derivative_in_delta(qx, h, T, delta):
    U, N = 3.0, 16
    m = oracle.make_model(U=U)
    eps = 1e-5
    num = (oracle.omega(m, N, qx, 0.0, h, T, delta + eps) -
           oracle.omega(m, N, qx, 0.0, h, T, delta - eps)) / (2 * eps)
    ana = _analytic_dOmega(oracle.RAGHU2, U, N, qx, 0.0, h, T, delta)
    assert abs(num - ana) <= 1e-5 * max(1.0, abs(ana))


def test_bcs_gap_equation_root_is_the_minimum():
    """Q = 0, h = 0: the minimum of Omega(Delta) solves the BCS gap equation
    1 = U/(4 N^2) sum_{k,eps} eta^2 tanh(R/2T) / R, found here by Brent's method."""
    from scipy.optimize import brentq

    U, T, N = 4.0, 0.005, 64
    p = oracle.RAGHU2
    m = oracle.make_model(U=U)
    ks = TWO_PI * np.arange(N) / N
    KX, KY = np.meshgrid(ks, ks)
    eta2 = (np.cos(KX) * np.cos(KY)).ravel() ** 2
    xi = np.concatenate([np.array([bands_eigvalsh(p, kx, ky) for kx, ky in
                                   zip(KX.ravel(), KY.ravel())])[:, b] - p["mu"] for b in range(2)])
    eta2b = np.concatenate([eta2, eta2])

    def gap_eq(d):
        R = np.sqrt(xi**2 + d * d * eta2b)
        return U / (4 * N * N) * np.sum(eta2b * np.tanh(R / (2 * T)) / R) - 1.0

    root = brentq(gap_eq, 1e-3, 0.2, xtol=1e-14)
    d_star, _, _ = search.golden_section(lambda d: oracle.omega(m, N, 0, 0, 0, T, d), 0.05, 0.2, 60)
    assert abs(d_star - root) < 2e-6
    # the 201-point grid of the N = 64 workload lands next to the root
    i, d_grid, _, om = search.minimize_grid(m, N, 0, 0, 0, T, 0.0, 0.2, 201)
    assert abs(d_grid - root) <= 0.2 / 200 / 2 + 1e-12
    assert om[i] < om[0]


def test_weak_coupling_is_normal_state():
    """With U = 2 the N = 64, T = 0.005 workload has its minimum at Delta = 0
    (the gap equation has no root: its right side stays below 1)."""
    m = oracle.make_model(U=2.0)
    i, d, _, om = search.minimize_grid(m, 64, 0, 0, 0, 0.005, 0.0, 0.2, 201)
    assert i == 0 and d == 0.0
    assert np.all(np.diff(om[:20]) > 0)


def test_per_band_coupling_gap_equations():
    """Each band with its own coupling U_eps (Sec. 2, V_eps per band): at Q = 0, h = 0 the minimum
    of the band's own Omega_eps(Delta) solves that band's gap equation
    1 = U_eps/(2 N^2) sum_k eta^2 tanh(R/2T) / R (Brent's method), and the two bands' minima differ.
    The coupling enters only through Delta^2/U_eps: Omega_eps(U_a) - Omega_eps(U_b) = N^2 Delta^2 (1/U_a - 1/U_b)."""
    from scipy.optimize import brentq

    U0, Ub, T, N = 4.0, (7.0, 3.0), 0.005, 48
    p = oracle.RAGHU2
    m = oracle.make_model(U=U0, U_band=Ub)
    ks = TWO_PI * np.arange(N) / N
    KX, KY = np.meshgrid(ks, ks)
    eta2 = (np.cos(KX) * np.cos(KY)).ravel() ** 2
    ev = np.array([bands_eigvalsh(p, kx, ky) for kx, ky in zip(KX.ravel(), KY.ravel())])
    roots = []
    for b in range(2):
        xi = ev[:, b] - p["mu"]

        def gap_eq(d, xi=xi, U=Ub[b]):
            R = np.sqrt(xi**2 + d * d * eta2)
            return U / (2 * N * N) * np.sum(eta2 * np.tanh(R / (2 * T)) / R) - 1.0

        root = brentq(gap_eq, 1e-3, 0.3, xtol=1e-14)
        d_star, _, _ = search.golden_section(lambda d, b=b: oracle.omega(m, N, 0, 0, 0, T, d, bands=True)[1][b],
                                             0.02, 0.3, 60)
        assert abs(d_star - root) < 2e-6, (b, d_star, root)
        roots.append(root)
    assert abs(roots[0] - roots[1]) > 0.01
    _, plain = oracle.omega(oracle.make_model(U=U0), N, 0.1, 0.0, 0.03, T, 0.07, bands=True)
    _, per = oracle.omega(m, N, 0.1, 0.0, 0.03, T, 0.07, bands=True)
    for b in range(2):
        want = N * N * 0.07**2 * (1 / Ub[b] - 1 / U0)
        assert abs((per[b] - plain[b]) - want) <= 1e-9 * abs(plain[b])
