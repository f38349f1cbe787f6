"""The numerical facts the FP32 k-sum and the band tables rely on, checked on the CPU.

Each test restates one claim made in the kernels' comments and checks it independently of them
(numpy, IEEE float32 / float64): where a shortcut gives the same bits as the full formula, and
where a truncated expansion stays inside its stated bound."""
import numpy as np
import pytest

ALPHA = [0.5, -0.125, 0.0625, -5.0 / 128.0, 7.0 / 256.0, -21.0 / 1024.0]  # sqrt(1+x) - 1 = sum alpha_n x^n


def f32_fma(a, b, c):
    """float32 fused multiply-add: the exact a*b + c, rounded once to float32."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def test_moment_series_of_R_minus_abs_s():
    """a = R - |s| = |s| sum_n alpha_n x^n, x = Delta^2 eta^2 / s^2, n <= 6, within 3.3e-8 of a
    for x <= 0.1 (the range the far-band moments take), and the coefficients are the binomial
    series of sqrt(1 + x) - 1."""
    from math import comb
    for n, a in enumerate(ALPHA, start=1):  # binomial(1/2, n) = (-1)^(n+1) C(2n, n) / (4^n (2n - 1))
        assert a == pytest.approx((-1) ** (n + 1) * comb(2 * n, n) / (4 ** n * (2 * n - 1)), rel=1e-15)
    x = np.linspace(0.0, 0.1, 10001)[1:]
    exact = np.sqrt(1.0 + x) - 1.0
    series = sum(a * x ** (n + 1) for n, a in enumerate(ALPHA))
    assert np.max(np.abs(series - exact) / exact) <= 3.3e-8
    # t = Delta^2 / Delta_max^2 <= 1 scales y = Delta_max^2 eta^2 / s^2: x = t y, moments |s| y^n
    rng = np.random.default_rng(1)
    s, y = rng.uniform(0.01, 3.0, 200), rng.uniform(0.0, 0.1, 200)  # the far bands of one item
    moments = [np.sum(s * y ** (n + 1)) for n in range(6)]
    for t in (0.0, 1e-3, 0.25, 0.7, 1.0):  # one output each
        via_moments = sum(ALPHA[n] * t ** (n + 1) * moments[n] for n in range(6))
        direct = np.sum(s * (np.sqrt(1.0 + t * y) - 1.0))
        assert via_moments == pytest.approx(direct, rel=3.3e-8, abs=1e-300)


@pytest.mark.parametrize("y", [26.0, 27.0, 40.0, 80.0])
def test_a_factor_below_2_to_minus_26_leaves_the_fp32_product_unchanged(y):
    """P + P e with e <= 2^-y, y >= 26, rounds to P in float32 for every P >= 1: the far form
    (threshold 27) and the one-exponential near form give the same bits as the full term."""
    rng = np.random.default_rng(int(y))
    P = np.float32(rng.uniform(1.0, 2.0 ** 32, 20000))
    P = np.concatenate([P, np.float32([1.0, 2.0, 4.0, np.nextafter(np.float32(2.0), np.float32(0.0))])])
    e = np.float32(2.0 ** -y)
    out = np.array([f32_fma(p, e, p) for p in P], dtype=np.float32)
    assert np.array_equal(out, P)
    # ... while 2^-22 would not (the bound is tight enough to matter)
    big = np.float32(2.0 ** -22)
    assert not np.array_equal(np.array([f32_fma(p, big, p) for p in P[:100]], dtype=np.float32), P[:100])


def test_fp64_negligible_exponentials_move_omega_below_fp64_rounding():
    """FP64 band terms take exp(-y) as 0 for y >= 40 (the k-sum's far bands need no exponential):
    the dropped -T ln(1 + q) is below 3 e^-40 T < 1.3e-17 T per band, so Omega per site (a mean of
    N^2 k-point terms) moves by less than 3.9e-17 T with three bands: for T <= 1 below a fifth of
    one FP64 ulp of a per-site value of 1."""
    rng = np.random.default_rng(40)
    T = rng.uniform(1e-4, 1.0, 20000)
    y1 = rng.uniform(40.0, 80.0, 20000)
    y2 = y1 + rng.uniform(0.0, 40.0, 20000)
    e1, e2 = np.exp(-y1), np.exp(-y2)
    q = e1 + e2 + e1 * e2
    assert np.all(T * np.log1p(q) < 1.3e-17 * T)
    assert 3.0 * 1.3e-17 < 0.2 * np.spacing(1.0)
    # a per-site mean of such terms moves by at most the largest of them
    terms = -T * np.log1p(q)
    assert abs(terms.mean()) < 1.3e-17
    # at y = 36 the dropped part of three bands would exceed half an ulp of 1 (the cut-off is not loose)
    assert 3.0 * np.exp(-36.0) > 0.5 * np.spacing(1.0)


def test_newton_steps_refine_fp32_eigenvalues_to_fp64():
    """Outer eigenvalues of a real symmetric 3x3 matrix from FP32 estimates and two Newton
    steps on det(A - x) = ((c2 - x) x - c1) x + c0, dividing by the derivative through an FP32
    reciprocal, the middle one from the trace: FP64 accuracy when the eigenvalues are at least
    1e-4 of the scale apart (the band tables fall back to FP64 Jacobi below that): the error of
    the cubic's roots grows like eps scale / gap, so ~1e-12 of the scale at the closest gaps
    and FP64 rounding for typical ones."""
    rng = np.random.default_rng(7)
    errs = []
    for _ in range(2000):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = np.sort(rng.uniform(-3.0, 3.0, 3))
        if np.min(np.diff(lam)) < 1e-4 * np.max(np.abs(lam)):
            continue
        A = q @ np.diag(lam) @ q.T
        A = 0.5 * (A + A.T)
        est = np.sort(np.linalg.eigvalsh(A.astype(np.float32)).astype(np.float64))  # ~1e-7 relative
        c2 = np.trace(A)
        c1 = A[0, 0] * A[1, 1] + A[0, 0] * A[2, 2] + A[1, 1] * A[2, 2] - A[0, 1] ** 2 - A[0, 2] ** 2 - A[1, 2] ** 2
        c0 = np.linalg.det(A)
        out = []
        for x in (est[0], est[2]):
            for _ in range(2):
                p = ((c2 - x) * x - c1) * x + c0
                dp = (2.0 * c2 - 3.0 * x) * x - c1
                x -= p * np.float64(np.float32(1.0) / np.float32(dp))
            out.append(x)
        e = np.array([out[0], c2 - out[0] - out[1], out[1]])
        ref = np.linalg.eigvalsh(A)
        errs.append(np.max(np.abs(e - ref)) / np.max(np.abs(ref)))
    assert max(errs) < 1e-11 and np.median(errs) < 1e-14, (max(errs), np.median(errs))


def _bands_app_a(kx, ky, t1=-1.0, t2=1.3, t3=-0.85, t4=-0.85):
    """App. A: the two eigenvalues of the 2 x 2 hopping matrix at (kx, ky), written out here."""
    cx, cy = np.cos(kx), np.cos(ky)
    t11 = -2.0 * (t1 * cx + t2 * cy) - 4.0 * t3 * cx * cy
    t22 = -2.0 * (t2 * cx + t1 * cy) - 4.0 * t3 * cx * cy
    t12 = -4.0 * t4 * np.sin(kx) * np.sin(ky)
    mean, root = 0.5 * (t11 + t22), np.sqrt((0.5 * (t11 - t22)) ** 2 + t12 ** 2)
    return mean - root, mean + root


@pytest.mark.parametrize("q", [(0.0, 0.0), (0.31, 0.0), (0.2, -0.13), (np.pi / 8, np.pi / 16)])
def test_minus_k_band_values_are_the_plus_k_values_relabelled(q):
    """The normal-state sums take the spin-down band values E(-k + Q/2) of the lattice as the
    spin-up values E(k + Q/2) relabelled k -> -k: on the N x N lattice (k = 2 pi (i, j) / N) the
    two multisets agree, so every lattice sum of a function of them agrees, here
    sum_k min(E - mu, -h), to FP64 rounding."""
    N, mu = 48, 1.54
    i = 2.0 * np.pi * np.arange(N) / N
    kx, ky = np.meshgrid(i, i, indexing="ij")
    up = np.concatenate([e.ravel() for e in _bands_app_a(kx + q[0] / 2, ky + q[1] / 2)]) - mu
    dn = np.concatenate([e.ravel() for e in _bands_app_a(-kx + q[0] / 2, -ky + q[1] / 2)]) - mu
    assert np.allclose(np.sort(up), np.sort(dn), rtol=0, atol=1e-13)
    for h in (0.0, 0.05, 0.15):
        a, b = np.sum(np.minimum(dn, -h)), np.sum(np.minimum(up, -h))
        assert abs(a - b) <= 1e-12 * abs(a)


def test_split_exponentials_equal_the_direct_exponentials():
    """FP64 near bands of a batch with one T: with P = R - d0 + h, M = R + d0 - h, the arguments
    {|R - |d||, R + |d|} / T (d = d0 - h) are {|P|, |M|} / T, and e^{-|P|/T} is e^{-alpha} e^{-eta}
    (P >= 0) or e^{alpha} e^{eta} (P < 0) with alpha = (R - d0)/T, eta = h/T (M likewise with
    beta = (R + d0)/T, -eta); arguments capped at 700 and |eta| <= 600 keep every factor taken
    finite; agreement with the direct exponentials within the arguments' own rounding."""
    rng = np.random.default_rng(64)
    n = 200000
    T = rng.uniform(1e-3, 0.05, n)
    h = rng.uniform(-0.2, 0.2, n)
    d0 = rng.uniform(-3.0, 3.0, n)
    R = np.abs(d0 - h) + rng.uniform(-40.0, 40.0, n) * T  # near: |R - |d|| / T < 40
    R = np.maximum(R, 0.0)
    d = d0 - h
    y = np.stack([np.abs(R - np.abs(d)), R + np.abs(d)]) / T
    direct = np.where(y < 40.0, np.exp(-np.minimum(y, 700.0)), 0.0)
    it = 1.0 / T
    al, be, eta = (R - d0) * it, (R + d0) * it, h * it
    assert np.all(np.abs(eta) <= 600.0)
    eam, eap = np.exp(np.minimum(-al, 700.0)), np.exp(np.minimum(al, 700.0))
    ebm, ebp = np.exp(np.minimum(-be, 700.0)), np.exp(np.minimum(be, 700.0))
    xp, xm = np.exp(eta), np.exp(-eta)
    ps, ms = al + eta, be - eta
    with np.errstate(over="ignore"):  # np.where forms both products; the unselected one may overflow
        e1 = np.where(ps >= 0.0, eam * xm, eap * xp)
        e2 = np.where(ms >= 0.0, ebm * xp, ebp * xm)
    e1 = np.where(np.abs(ps) >= 40.0, 0.0, e1)
    e2 = np.where(np.abs(ms) >= 40.0, 0.0, e2)
    assert np.all(np.isfinite(e1)) and np.all(np.isfinite(e2))
    split = np.sort(np.stack([e1, e2]), axis=0)
    want = np.sort(direct, axis=0)
    both = np.all(np.abs(np.sort(np.stack([np.abs(ps), np.abs(ms)]), axis=0) - np.sort(y, axis=0)) < 1e-9, axis=0)
    both &= np.all(np.abs(np.sort(y, axis=0) - 40.0) > 1e-6, axis=0)  # away from the cut-off
    scale = (np.abs(al) + np.abs(eta) + np.abs(be) + 1.0) * 2.3e-16
    assert np.all(np.abs(split - want)[:, both] <= 8.0 * scale[both] * np.maximum(want[:, both], 1e-300) + 1e-300)


def test_two_log_factors_under_one_log1p():
    """log1p(q0) + log1p(q1) = log1p(q0 + q1 + q0 q1) (the FP64 flush puts a lane's two near
    entries under one logarithm), to a few FP64 ulp, for q from 1e-18 (a factor e^-40) to 3."""
    rng = np.random.default_rng(3)
    q0 = np.concatenate([10.0 ** rng.uniform(-18, np.log10(3.0), 50000), [0.0, 3.0]])
    q1 = np.concatenate([10.0 ** rng.uniform(-18, np.log10(3.0), 50000), [5e-18, 0.0]])
    lhs = np.log1p(q0) + np.log1p(q1)
    rhs = np.log1p(q0 + q1 + q0 * q1)
    assert np.all(np.abs(lhs - rhs) <= 4.0 * np.spacing(np.maximum(lhs, 1e-300)) + 1e-300)
