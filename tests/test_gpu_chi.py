"""Static Cooper pair susceptibility (App. C) on the GPU vs the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from oracle import chi as ochi
from paper_1412_8754_gb300 import ffe

pytestmark = pytest.mark.gpu


def test_two_band_chi_vs_oracle():
    m = oracle.make_model()
    N = 24
    qs = [(0.0, 0.0), (0.5, 0.0), (1.1, -0.4), (4 * math.pi / N, 0.0)]
    with ffe.Context(prec=ffe.FFE_FP64, eta_amp=4.0) as c:
        for h, T in [(0.0, 0.02), (0.08, 0.005), (0.15, 1e-4)]:
            got = c.pair_susceptibility(N, [q[0] for q in qs], [q[1] for q in qs], h, T)
            assert got.shape == (len(qs), 2, 2)
            for i, (qx, qy) in enumerate(qs):
                ref = ochi.chi(m, N, qx, qy, h, T, eta_amp=4.0)
                np.testing.assert_allclose(got[i], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_three_band_chi_vs_oracle():
    N = 16
    qx = np.array([0.0, 0.2, 0.6])
    qy = np.array([0.0, 0.0, 0.3])
    with ffe.Context(prec=ffe.FFE_FP64, eta_amp=4.0, model="daghofer3", U=1.2) as c:
        for h, T in [(0.0, 0.002), (0.025, 1e-4)]:
            got = c.pair_susceptibility(N, qx, qy, h, T)
            assert got.shape == (3, 3, 3)
            for i in range(3):
                ref = ochi.chi("daghofer3", N, qx[i], qy[i], h, T, eta_amp=4.0)
                np.testing.assert_allclose(got[i], ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())


def test_chi_rejects_bad_arguments():
    with ffe.Context(prec=ffe.FFE_FP64) as c:
        with pytest.raises(ffe.FFEError):
            c.pair_susceptibility(7, [0.0], [0.0], 0.0, 0.01)
        with pytest.raises(ffe.FFEError):
            c.pair_susceptibility(8, [0.0], [0.0], 0.0, 0.0)
