"""FP64 oracle of the static Cooper pair susceptibility of App. C (test infrastructure only).

  chi_{e e'}(q) = -(1/N^2) sum_k eta(-k-q)^2 [f(-E_{e,k,up}) - f(E_{e',-k-q,down})]
                                             / (0 - E_{e,k,up} - E_{e',-k-q,down})
with E_{e,k,up} = E_e(k) - mu - h, E_{e',-k-q,down} = E_e'(-k-q) - mu + h, f the
Fermi function and eta the s+- structure factor eta_amp cos kx cos ky (App. C
uses eta_amp = 4).  Band energies: the two-band closed form (App. A) or the
three-band model's eigenvalues (App. B, oracle.threeband); the summand and the
k-sum are the C routine ffeo_chi_given.  `eta_at="relative"` evaluates eta at
k + q/2 instead -- the free energy's convention -- for the pin that relates chi
to the curvature of Omega at Delta = 0 (tests/test_oracle_chi.py).
"""
from __future__ import annotations

import numpy as np

from . import _dp, band_energies, lib
from . import threeband as tb


def _bands(model, kx, ky):
    """[..., nb] band energies at (kx, ky): model is an oracle.Model (two bands) or "daghofer3"."""
    if isinstance(model, str):
        return tb.band_energies(kx, ky)
    kx, ky = np.broadcast_arrays(np.asarray(kx, float), np.asarray(ky, float))
    out = np.array([band_energies(model, a, b) for a, b in zip(kx.ravel(), ky.ravel())])
    return out.reshape(kx.shape + (2,))


def chi(model, N: int, qx: float, qy: float, h: float, T: float, eta_amp: float = 4.0, mu=None,
        eta_at: str = "down") -> np.ndarray:
    """chi[nb, nb] at pair momentum q (App. C convention: spin up at k, spin down at -k-q)."""
    k = 2.0 * np.pi * np.arange(N) / N
    KY, KX = np.meshgrid(k, k, indexing="ij")
    e_up = np.ascontiguousarray(_bands(model, KX, KY)).reshape(N * N, -1)
    e_dn = np.ascontiguousarray(_bands(model, -KX - qx, -KY - qy)).reshape(N * N, -1)
    nb = e_up.shape[1]
    if eta_at == "down":
        ex, ey = -KX - qx, -KY - qy
    elif eta_at == "relative":
        ex, ey = KX + qx / 2, KY + qy / 2
    else:
        raise ValueError(eta_at)
    eta2 = np.ascontiguousarray((eta_amp * np.cos(ex) * np.cos(ey)).ravel() ** 2)
    if mu is None:
        mu = tb.DAGHOFER3["mu"] if isinstance(model, str) else model.mu
    out = np.zeros(nb * nb)
    lib().ffeo_chi_given(nb, N, _dp(e_up), _dp(e_dn), _dp(eta2), mu, h, T, _dp(out))
    return out.reshape(nb, nb)
