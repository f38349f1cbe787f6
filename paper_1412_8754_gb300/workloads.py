"""Seeded synthetic inputs of the workloads (shared by tests, bench and oracle runs).

This module holds parameter lists only -- no arithmetic of the method.  The
paper measures on synthetic model parameters, not on a dataset: one q vector,
200 Delta values on an N x N lattice of the two-band model (Sec. 3,
performance evaluation).  The workloads below keep that shape and scale it up:

  small_bcs     N=64, Q=0, h=0, T=0.005, 201 Delta in [0, 0.2]; U=2 (normal
                state) and U=4 (interior BCS minimum)
  fflo_scan     N=1024, 64 q in [0, 0.2 pi] along x, 32 h in [0, 0.15],
                T=0.002, 256 Delta in [0, 0.2]
  uneven_jobs   512 jobs, N uniform over {256, 512, 1024, 2048}, (q, h, T)
                uniform in [0, 0.2 pi] x [0, 0.15] x [0.001, 0.02], Delta grid
                of 32..256 points on [0, 0.2] (numpy default_rng(1234))
  surrogate_set (q, h, T, Delta) samples for the surrogate (default_rng(1235))
  phase_diagram N=2048, 64 h in [0, 0.15] x 64 T in [0.001, 0.03], 64 q,
                golden-section search with 24 reductions on [0, 0.2]
  ff_scan       a scan that reaches the FF phase: the same hoppings with
                mu = 3.8 (small hole pockets around (pi, pi), where
                eta = cos kx cos ky is close to 1) and U = 5; 31 q in
                [0, 0.3] along x, 11 h in [0.03, 0.05], T in {0.002, 0.003},
                41 Delta in [0, 0.1]: BCS, FF and normal points
"""
from __future__ import annotations

import math

import numpy as np

RAGHU2 = dict(t1=-1.0, t2=1.3, t3=-0.85, t4=-0.85, mu=1.54)  # App. A

SMALL_BCS = dict(N=64, qx=[0.0], qy=[0.0], h=[0.0], T=[0.005], lo=0.0, hi=0.2, n=201)


def fflo_scan(N=1024, n_q=64, n_h=32, n_delta=256, T=0.002):
    return dict(N=N, qx=np.linspace(0.0, 0.2 * math.pi, n_q), qy=np.zeros(n_q),
                h=np.linspace(0.0, 0.15, n_h), T=np.array([T]), lo=0.0, hi=0.2, n=n_delta)


FF_MODEL = dict(mu=3.8, U=5.0)


def ff_scan(N=64, n_q=31, n_h=11, n_delta=41, T=(0.002, 0.003)):
    return dict(N=N, qx=np.linspace(0.0, 0.3, n_q), qy=np.zeros(n_q), h=np.linspace(0.03, 0.05, n_h),
                T=np.array(T, dtype=float), lo=0.0, hi=0.1, n=n_delta)


def threeband_scan(N=1024, n_q=16, n_h=16, n_delta=64, T=0.001):
    """Phase scan of the three-band model (App. B, eV): q along x in [0, 0.1 pi], h in
    [0, 0.03], Delta in [0, 0.05]; with U = 1.2 eV the gap is ~0.02 eV at h = 0 and the
    Pauli limit near h = 0.014 eV."""
    return dict(N=N, qx=np.linspace(0.0, 0.1 * math.pi, n_q), qy=np.zeros(n_q),
                h=np.linspace(0.0, 0.03, n_h), T=np.array([T]), lo=0.0, hi=0.05, n=n_delta, U=1.2)


def uneven_jobs(n_jobs=512, seed=1234, sizes=(256, 512, 1024, 2048)):
    rng = np.random.default_rng(seed)
    N = rng.choice(np.array(sizes), size=n_jobs)
    q = rng.uniform(0.0, 0.2 * math.pi, n_jobs)
    h = rng.uniform(0.0, 0.15, n_jobs)
    T = rng.uniform(0.001, 0.02, n_jobs)
    n = rng.integers(32, 257, n_jobs)
    return dict(N=N.astype(np.int32), qx=q, qy=np.zeros(n_jobs), h=h, T=T,
                lo=np.zeros(n_jobs), hi=np.full(n_jobs, 0.2), n=n.astype(np.int32))


def surrogate_set(n_groups=8192, n_ht=16, n_delta=16, seed=1235, T_hi=0.03):
    """Training samples of the surrogate, uniform over the scan box:
    q per group, (h, T) pairs per group, Delta values per (q, h, T) line with
    Delta = 0 first (the reference of the condensation energy).
    Returns arrays of shape [n_groups], [n_groups, n_ht], [n_groups, n_ht, n_delta]."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.0, 0.2 * math.pi, n_groups)
    h = rng.uniform(0.0, 0.15, (n_groups, n_ht))
    T = rng.uniform(0.001, T_hi, (n_groups, n_ht))
    d = rng.uniform(0.0, 0.2, (n_groups, n_ht, n_delta))
    d[..., 0] = 0.0
    return dict(q=q, h=h, T=T, delta=d)


SURROGATE_SHIFT = np.array([0.0, 0.0, 0.001, 0.0])
SURROGATE_SCALE = 1.0 / np.array([0.2 * math.pi, 0.15, 0.029, 0.2])


def phase_diagram(N=2048, n_q=64, n_h=64, n_T=64, steps=24):
    return dict(N=N, qx=np.linspace(0.0, 0.2 * math.pi, n_q), qy=np.zeros(n_q),
                h=np.linspace(0.0, 0.15, n_h), T=np.linspace(0.001, 0.03, n_T), lo=0.0, hi=0.2, n=steps)


def random_points(n, seed=0, Ns=(8, 16, 24, 32, 64), qmax=0.2 * math.pi, hmax=0.15,
                  Tlo=0.001, Thi=0.03, dmax=0.2):
    rng = np.random.default_rng(seed)
    return dict(N=rng.choice(np.array(Ns), size=n).astype(np.int32), qx=rng.uniform(-qmax, qmax, n),
                qy=rng.uniform(-qmax / 4, qmax / 4, n), h=rng.uniform(-hmax, hmax, n),
                T=rng.uniform(Tlo, Thi, n), delta=rng.uniform(0.0, dmax, n))
