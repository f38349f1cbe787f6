"""Delta search and phase labelling of the FP64 oracle (test infrastructure only).

Alg. 1 of the paper: for each pair momentum q, scan Delta, keep the Delta with
the lowest Omega; then keep the q with the lowest Omega.  The readings used
where the paper leaves the details open:

* Delta grid: inclusive ``numpy.linspace(lo, hi, n)``.  Argmin = lowest Omega,
  exact ties go to the lowest index (``numpy.argmin`` semantics).
* Golden-section search on [lo, hi] with phi = (sqrt 5 - 1)/2: interior points
  x1 = a + (1-phi)(b-a), x2 = a + phi(b-a); keep [a, x2] when
  Omega(x1) <= Omega(x2), else [x1, b]; ``n_steps`` reductions, each followed
  by one new evaluation.  Delta = lo is evaluated as well (it is the normal
  state and a legitimate minimum).  The result is the lowest Omega among all
  evaluated points, ties going to the smaller Delta.
* Phase label per (h, T): Omega_N = Omega(q=0, Delta=0).  A q is a
  superconducting candidate when Omega(q, Delta*_q) < Omega(q, 0) - tau; the
  label is NORMAL unless the best candidate (ties -> lowest q index) has
  Omega < Omega_N - tau, then BCS if its q is zero, else FFLO (the FF phase of
  Sec. 2).  tau = 1e-12 |Omega_N| is the FP64 tie band.
"""
from __future__ import annotations

import math
from typing import Callable, Sequence

import numpy as np

from . import Model, omega_batch

NORMAL, BCS, FFLO = 0, 1, 2
PHI = (math.sqrt(5.0) - 1.0) / 2.0
TAU_REL = 1e-12


def delta_grid(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n)


def grid_argmin(values: Sequence[float]) -> int:
    """Lowest value, exact ties to the lowest index."""
    v = np.asarray(values, dtype=np.float64)
    best = 0
    for i in range(1, v.size):
        if v[i] < v[best]:
            best = i
    return best


def golden_points(lo: float, hi: float):
    a, b = lo, hi
    return a + (1.0 - PHI) * (b - a), a + PHI * (b - a)


def golden_section(f: Callable[[float], float], lo: float, hi: float, n_steps: int):
    """Returns (delta_star, f_star, evaluated list of (delta, f)) for a scalar f."""
    a, b = lo, hi
    x1, x2 = golden_points(a, b)
    f1, f2 = f(x1), f(x2)
    seen = [(lo, f(lo)), (x1, f1), (x2, f2)]
    for _ in range(n_steps):
        if f1 <= f2:
            b, x2, f2 = x2, x1, f1
            x1 = a + (1.0 - PHI) * (b - a)
            f1 = f(x1)
            seen.append((x1, f1))
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + PHI * (b - a)
            f2 = f(x2)
            seen.append((x2, f2))
    best = seen[0]
    for x, v in seen[1:]:
        if v < best[1] or (v == best[1] and x < best[0]):
            best = (x, v)
    return best[0], best[1], seen


def golden_section_batch(evaluate: Callable[[np.ndarray], np.ndarray], lo, hi, n_steps: int,
                         trace: bool = False):
    """Lockstep golden-section search for many independent points.

    ``evaluate(deltas[n]) -> omegas[n]`` evaluates each point at its own Delta.
    Returns (delta_star[n], omega_star[n], omega_lo[n]).  With ``trace`` it also
    returns a dict of the search's history: ``x`` and ``f`` [3 + n_steps, n], the
    evaluated Delta and Omega in order (lo, x1, x2, then one per reduction);
    ``a``, ``b`` and ``margin`` [n_steps, n], the bracket before each reduction
    and |Omega(x1) - Omega(x2)| of the comparison that decides it.  Up to the
    first comparison whose margin is below twice a per-value error bound, any
    evaluation within that bound of these values takes the same decisions."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    a, b = lo.copy(), hi.copy()
    x1 = a + (1.0 - PHI) * (b - a)
    x2 = a + PHI * (b - a)
    f0 = evaluate(lo.copy())
    f1 = evaluate(x1.copy())
    f2 = evaluate(x2.copy())
    best_x, best_f = lo.copy(), f0.copy()
    tr = dict(x=[lo.copy(), x1.copy(), x2.copy()], f=[f0, f1, f2], a=[], b=[], margin=[])

    def take(x, fx):
        better = (fx < best_f) | ((fx == best_f) & (x < best_x))
        best_x[better] = x[better]
        best_f[better] = fx[better]

    take(x1, f1)
    take(x2, f2)
    for _ in range(n_steps):
        tr["a"].append(a)
        tr["b"].append(b)
        tr["margin"].append(np.abs(f1 - f2))
        left = f1 <= f2                      # keep [a, x2], else keep [x1, b]
        a, b = np.where(left, a, x1), np.where(left, x2, b)
        newx = np.where(left, a + (1.0 - PHI) * (b - a), a + PHI * (b - a))
        fn = evaluate(newx.copy())
        x1, f1, x2, f2 = (np.where(left, newx, x2), np.where(left, fn, f2),
                          np.where(left, x1, newx), np.where(left, f1, fn))
        take(newx, fn)
        tr["x"].append(newx)
        tr["f"].append(fn)
    if not trace:
        return best_x, best_f, f0
    shape = (0,) + lo.shape
    tr = {k: (np.stack(v) if v else np.zeros(shape)) for k, v in tr.items()}
    return best_x, best_f, f0, tr


def phase_label(omega_star: Sequence[float], omega_zero: Sequence[float],
                q_is_zero: Sequence[bool], tau_rel: float = TAU_REL):
    """Label one (h, T) point from the per-q minima.  Returns (label, q_index or -1)."""
    ws = np.asarray(omega_star, dtype=np.float64)
    w0 = np.asarray(omega_zero, dtype=np.float64)
    qz = np.asarray(q_is_zero, dtype=bool)
    zero_idx = np.flatnonzero(qz)
    if zero_idx.size == 0:
        raise ValueError("phase labels need q = 0 in the q list")
    omega_n = w0[zero_idx[0]]
    tau = tau_rel * abs(omega_n)
    best = -1
    for i in range(ws.size):
        if ws[i] < w0[i] - tau and (best < 0 or ws[i] < ws[best]):
            best = i
    if best < 0 or not (ws[best] < omega_n - tau):
        return NORMAL, -1
    return (BCS if qz[best] else FFLO), best


def minimize_grid(model: Model, N: int, qx: float, qy: float, h: float, T: float,
                  lo: float, hi: float, n: int, nthreads: int = 0):
    """Alg. 1 inner loop on one parameter point: Omega over the Delta grid and its argmin."""
    d = delta_grid(lo, hi, n)
    om, _, _ = omega_batch(model, N, qx, qy, h, T, d, nthreads=nthreads)
    i = grid_argmin(om)
    return i, d[i], om[i], om
