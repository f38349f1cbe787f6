"""FP64 oracle of the three-band model of App. B (test infrastructure only).

The hopping matrix T(k) of App. B is a 3x3 Hermitian matrix (d_xz, d_yz,
d_xy orbitals):
  T11 = 2 t2 cos kx + 2 t1 cos ky + 4 t3 cos kx cos ky
        + 2 t11 (cos 2kx - cos 2ky) + 4 t12 cos 2kx cos 2ky
  T22 = 2 t1 cos kx + 2 t2 cos ky + 4 t3 cos kx cos ky
        - 2 t11 (cos 2kx - cos 2ky) + 4 t12 cos 2kx cos 2ky
  T33 = eps0 + 2 t5 (cos kx + cos ky) + 4 t6 cos kx cos ky
        + 2 t9 (cos 2kx + cos 2ky) + 4 t10 (cos 2kx cos ky + cos kx cos 2ky)
  T12 = T21 = 4 t4 sin kx sin ky
  T13 = conj(T31) = 2i t7 sin kx + 4i t8 sin kx cos ky
  T23 = conj(T32) = 2i t7 sin ky + 4i t8 sin ky cos kx
Its eigenvalues (numpy.linalg.eigvalsh, a library step, ascending: bands
0, 1, 2) at k + Q/2 and -k + Q/2 enter the same free energy as the
two-band model (Sec. 2, Eq. freeene), summed over three bands by the C
oracle (ffeo_omega_given).  Energies in eV.  Pinned in
tests/test_oracle_threeband.py by the printed filling (n = 4 at
mu = 0.4748), by trace and determinant of the printed matrix, by the
lattice symmetries and by the Delta = 0 and T -> 0 limits.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _dp, lib

# App. B, hopping parameters in eV and the chemical potential of n = 4
DAGHOFER3 = dict(t1=-0.08, t2=0.1825, t3=0.08375, t4=-0.03, t5=0.15, t6=0.15, t7=-0.12, t8=0.06,
                 t9=0.0, t10=-0.024, t11=-0.01, t12=0.0275, eps0=0.75, mu=0.4748)


def hopping_matrix(kx, ky, p=DAGHOFER3):
    """T(k) of App. B, shape [..., 3, 3] complex."""
    kx, ky = np.broadcast_arrays(np.asarray(kx, float), np.asarray(ky, float))
    cx, cy, sx, sy = np.cos(kx), np.cos(ky), np.sin(kx), np.sin(ky)
    c2x, c2y = np.cos(2 * kx), np.cos(2 * ky)
    T = np.zeros(kx.shape + (3, 3), dtype=complex)
    T[..., 0, 0] = (2 * p["t2"] * cx + 2 * p["t1"] * cy + 4 * p["t3"] * cx * cy
                    + 2 * p["t11"] * (c2x - c2y) + 4 * p["t12"] * c2x * c2y)
    T[..., 1, 1] = (2 * p["t1"] * cx + 2 * p["t2"] * cy + 4 * p["t3"] * cx * cy
                    - 2 * p["t11"] * (c2x - c2y) + 4 * p["t12"] * c2x * c2y)
    T[..., 2, 2] = (p["eps0"] + 2 * p["t5"] * (cx + cy) + 4 * p["t6"] * cx * cy
                    + 2 * p["t9"] * (c2x + c2y) + 4 * p["t10"] * (c2x * cy + cx * c2y))
    T[..., 0, 1] = T[..., 1, 0] = 4 * p["t4"] * sx * sy
    T[..., 0, 2] = 2j * p["t7"] * sx + 4j * p["t8"] * sx * cy
    T[..., 1, 2] = 2j * p["t7"] * sy + 4j * p["t8"] * sy * cx
    T[..., 2, 0] = np.conj(T[..., 0, 2])
    T[..., 2, 1] = np.conj(T[..., 1, 2])
    return T


def band_energies(kx, ky, p=DAGHOFER3):
    """Eigenvalues of T(k), ascending, shape [..., 3]."""
    return np.linalg.eigvalsh(hopping_matrix(kx, ky, p))


def band_grids(N: int, qx: float, qy: float, p=DAGHOFER3):
    """(E(k + Q/2), E(-k + Q/2)) on the lattice k = 2 pi (i, j)/N, each [N, N, 3] indexed [j, i, band]."""
    k = 2.0 * np.pi * np.arange(N) / N
    KY, KX = np.meshgrid(k, k, indexing="ij")
    return (np.ascontiguousarray(band_energies(KX + qx / 2, KY + qy / 2, p)),
            np.ascontiguousarray(band_energies(-KX + qx / 2, -KY + qy / 2, p)))


def omega_batch(N: int, qx: float, qy: float, h, T, delta, U: float, eta_amp: float = 1.0, p=DAGHOFER3,
                bands: bool = False, nthreads: int = 0, U_band=(0.0, 0.0, 0.0)):
    """Omega of the three-band model at many (h, T, Delta) of one (N, Q); U_band[b] > 0 is band
    b's own coupling (else U).

    Returns (omega[n], omega_band[n, 3] or None, threads_used)."""
    e_up, e_dn = band_grids(N, qx, qy, p)
    h, T, delta = (np.ascontiguousarray(a, dtype=np.float64).ravel()
                   for a in np.broadcast_arrays(np.asarray(h, float), np.asarray(T, float),
                                                np.asarray(delta, float)))
    n = h.size
    om = np.zeros(n)
    ob = np.zeros((n, 3)) if bands else None
    L = lib()
    Ub = np.array([u if u > 0.0 else U for u in U_band], dtype=np.float64)
    used = L.ffeo_omega_given_batch(3, N, _dp(e_up), _dp(e_dn), eta_amp, p["mu"], _dp(Ub), n, _dp(h), _dp(T),
                                    _dp(delta), _dp(om), _dp(ob) if bands else None, int(nthreads))
    return om, ob, used


def filling(N: int, mu: float, p=DAGHOFER3) -> float:
    """Electrons per site at T = 0, h = 0: two spins times the fraction of (k, band) states below mu."""
    e, _ = band_grids(N, 0.0, 0.0, p)
    return 2.0 * float(np.count_nonzero(e < mu)) / (N * N)
