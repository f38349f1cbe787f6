"""Pins of the oracle's Delta search and phase labelling (Alg. 1)."""
import math

import numpy as np
import pytest

from oracle import search

RNG = np.random.default_rng(7)


def test_grid_argmin_matches_numpy_first_occurrence():
    for _ in range(200):
        v = RNG.integers(0, 5, size=RNG.integers(1, 40)).astype(float)
        assert search.grid_argmin(v) == int(np.argmin(v))


def test_delta_grid_is_inclusive_linspace():
    g = search.delta_grid(0.0, 0.2, 201)
    assert g[0] == 0.0 and g[-1] == 0.2 and len(g) == 201
    assert abs(g[1] - 0.001) < 1e-15


def test_golden_converges_to_vertex_within_final_bracket():
    for c in RNG.uniform(0.01, 0.19, 20):
        n = 24
        x, fx, seen = search.golden_section(lambda d: (d - c) ** 2, 0.0, 0.2, n)
        assert len(seen) == n + 3
        assert abs(x - c) <= 0.2 * search.PHI ** (n + 1)


def test_golden_keeps_lower_endpoint():
    x, fx, _ = search.golden_section(lambda d: d * d + 1.0, 0.0, 0.2, 24)
    assert x == 0.0 and fx == 1.0


def test_golden_decreasing_function_reaches_upper_end():
    n = 30
    x, _, _ = search.golden_section(lambda d: -d, 0.0, 0.2, n)
    assert 0.2 - x <= 0.2 * search.PHI ** (n + 1)


def test_golden_bracket_shrinks_by_phi():
    """After each reduction the bracket is phi times shorter (exact arithmetic)."""
    a, b = 0.0, 1.0
    x1, x2 = search.golden_points(a, b)
    assert math.isclose(x2 - a, search.PHI * (b - a))
    assert math.isclose(b - x1, search.PHI * (b - a))
    # the retained interior point is again a golden point of the new bracket
    assert math.isclose(x1 - a, search.PHI * (x2 - a))


def test_golden_batch_equals_scalar():
    cs = RNG.uniform(0.0, 0.2, 16)
    ws = RNG.uniform(-1, 1, 16)

    def f_scalar(i):
        return lambda d: (d - cs[i]) ** 2 * (1 + ws[i] * d) + 0.3 * math.sin(40 * d) * 1e-3

    def f_batch(d):
        return np.array([f_scalar(i)(d[i]) for i in range(len(d))])

    xb, fb, f0 = search.golden_section_batch(f_batch, np.zeros(16), np.full(16, 0.2), 24)
    for i in range(16):
        x, fx, _ = search.golden_section(f_scalar(i), 0.0, 0.2, 24)
        assert xb[i] == x and fb[i] == fx
        assert f0[i] == f_scalar(i)(0.0)


@pytest.mark.parametrize("ws,w0,qz,label,q", [
    ([-10.0, -10.0, -10.0], [-10.0, -10.0, -10.0], [1, 0, 0], search.NORMAL, -1),
    ([-10.5, -10.2, -10.0], [-10.0, -10.0, -10.0], [1, 0, 0], search.BCS, 0),
    ([-10.5, -10.7, -10.6], [-10.0, -10.0, -10.0], [1, 0, 0], search.FFLO, 1),
    ([-10.0, -10.7, -10.7], [-10.0, -10.0, -10.0], [1, 0, 0], search.FFLO, 1),   # tie -> lowest q
    # a q whose own normal state is lower but which does not beat Omega_N is normal
    ([-10.0, -9.99, -9.0], [-10.0, -9.98, -9.0], [1, 0, 0], search.NORMAL, -1),
    # inside the FP64 tie band: not a candidate
    ([-10.0 - 1e-13, -10.0, -10.0], [-10.0, -10.0, -10.0], [1, 0, 0], search.NORMAL, -1),
])
def test_phase_label_cases(ws, w0, qz, label, q):
    assert search.phase_label(ws, w0, np.array(qz, bool)) == (label, q)


def test_phase_label_needs_q_zero():
    with pytest.raises(ValueError):
        search.phase_label([-1.0], [-1.0], [False])


def test_golden_trace_of_a_parabola():
    """On f = (x - c)^2 the traced history is the scalar search's: the same evaluated points in
    order, brackets that shrink by phi and always contain c, and decision margins
    |f(x1) - f(x2)| = |x1 - x2| |x1 + x2 - 2c| of the bracket's interior points."""
    c, n = 0.0731, 12
    xb, fb, f0, tr = search.golden_section_batch(lambda d: (d - c) ** 2, np.zeros(1), np.full(1, 0.2), n,
                                                 trace=True)
    x, fx, seen = search.golden_section(lambda d: (d - c) ** 2, 0.0, 0.2, n)
    assert xb[0] == x and [s[0] for s in seen] == list(tr["x"][:, 0])
    assert tr["x"].shape == (n + 3, 1) and tr["margin"].shape == (n, 1)
    w = tr["b"][:, 0] - tr["a"][:, 0]
    np.testing.assert_allclose(w[1:] / w[:-1], search.PHI, rtol=1e-9)
    assert np.all((tr["a"][:, 0] <= c) & (c <= tr["b"][:, 0]))
    for k in range(n):
        a, b = tr["a"][k, 0], tr["b"][k, 0]
        x1, x2 = a + (1 - search.PHI) * (b - a), a + search.PHI * (b - a)
        assert math.isclose(tr["margin"][k, 0], abs(x1 - x2) * abs(x1 + x2 - 2 * c), rel_tol=1e-6, abs_tol=1e-18)


def test_golden_trace_flags_a_flat_function():
    """A constant function makes every decision a tie: margin 0."""
    _, _, _, tr = search.golden_section_batch(lambda d: np.ones_like(d), np.zeros(3), np.full(3, 0.2), 8, trace=True)
    assert np.all(tr["margin"] == 0.0)
