"""ffe_omega_noalloc: Omega with every intermediate in the library's fixed
device array, for callers that cannot allocate device memory at call time
(a process whose free device memory belongs to its own pool, or a loop where
a cudaMalloc would synchronise the device).  Its results must equal those of
ffe_omega, the allocating entry point, on two calls in a row, and the
oracle's, within the per-site tolerance of the parity tests; the largest call
the array takes (N = 2048, 512 points) is checked too.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1412_8754_gb300 import ffe

pytestmark = pytest.mark.gpu

TOL = {ffe.FFE_FP64: 1e-9, ffe.FFE_FP32C: 2e-7}  # per lattice site, as for ffe_omega


def _model(prec, U, eta=1.0):
    return ffe.ffe_model(ffe.FFE_MODEL_RAGHU2, prec, -1.0, 1.3, -0.85, -0.85, 1.54, U, eta)


def _noalloc(model, N, qx, qy, h, T, d):
    import torch

    dev = torch.device("cuda")
    th, tT, td = (torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev) for a in (h, T, d))
    out = torch.full((len(h),), 12345.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    st = ffe.lib().ffe_omega_noalloc(ctypes.byref(model), N, qx, qy, ctypes.c_void_p(th.data_ptr()),
                                     ctypes.c_void_p(tT.data_ptr()), ctypes.c_void_p(td.data_ptr()), len(h),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == ffe.FFE_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", [ffe.FFE_FP32C, ffe.FFE_FP64])
def test_noalloc_matches_ffe_omega_on_two_calls(prec):
    rng = np.random.default_rng(77)
    U, eta = 3.0, 1.0
    model = _model(prec, U, eta)
    calls = [(128, 0.37, 0.0, 300), (64, 0.12, -0.05, 45)]  # ragged sizes, different N, Q
    with ffe.Context(prec=prec, U=U, eta_amp=eta) as ctx:
        for N, qx, qy, n in calls:
            h = rng.uniform(-0.15, 0.15, n)
            T = rng.uniform(0.001, 0.03, n)
            d = rng.uniform(0.0, 0.2, n)
            got = _noalloc(model, N, qx, qy, h, T, d)
            ref = ctx.omega(ffe.points(N, qx, qy, h, T, d))
            err = np.abs(got - ref) / N**2
            assert np.all(np.isfinite(got))
            assert err.max() <= TOL[prec], err.max()


@pytest.mark.parametrize("prec", [ffe.FFE_FP32C, ffe.FFE_FP64])
def test_noalloc_matches_the_oracle(prec):
    """Ragged lattice (N = 24: 576 k-points), 77 points (three batches, the last ragged), both
    signs of h, low and high T (far and near bands), against the oracle directly."""
    rng = np.random.default_rng(78)
    U, N, qx, qy, n = 4.0, 24, 0.21, -0.07, 77
    h = rng.uniform(-0.12, 0.12, n)
    T = np.where(np.arange(n) % 2 == 0, 0.002, rng.uniform(0.005, 0.05, n))
    d = rng.uniform(0.0, 0.2, n)
    got = _noalloc(_model(prec, U), N, qx, qy, h, T, d)
    ref, _, _ = oracle.omega_batch(oracle.make_model(U=U), N, qx, qy, h, T, d)
    assert (np.abs(got - ref) / N**2).max() <= TOL[prec]


def test_noalloc_at_the_array_limits():
    """The largest call the fixed array holds (N = 2048, 512 points: the normal-state items and
    the k-sum items at their caps), against ffe_omega and, on a few points, the oracle."""
    rng = np.random.default_rng(79)
    U, N, qx, n = 4.0, 2048, 0.3, 512
    h = rng.uniform(0.0, 0.15, n)
    T = rng.uniform(0.001, 0.03, n)
    d = rng.uniform(0.0, 0.2, n)
    prec = ffe.FFE_FP32C
    got = _noalloc(_model(prec, U), N, qx, 0.0, h, T, d)
    again = _noalloc(_model(prec, U), N, qx, 0.0, h, T, d)
    assert np.array_equal(got, again)
    with ffe.Context(prec=prec, U=U) as ctx:
        ref = ctx.omega(ffe.points(N, qx, 0.0, h, T, d))
    assert (np.abs(got - ref) / N**2).max() <= TOL[prec]
    pick = np.array([0, 31, 32, 255, 256, 511])
    orc, _, _ = oracle.omega_batch(oracle.make_model(U=U), N, qx, 0.0, h[pick], T[pick], d[pick])
    assert (np.abs(got[pick] - orc) / N**2).max() <= TOL[prec]


def test_noalloc_flags_invalid_points_on_the_device():
    """T <= 0 or a non-finite input cannot be seen on the host (device arrays): such a point gets
    Omega = NaN, the others are computed as usual."""
    U, N = 3.0, 32
    h = np.array([0.01, 0.02, 0.03, 0.04, np.nan])
    T = np.array([0.01, 0.0, -0.01, 0.01, 0.01])
    d = np.array([0.05, 0.05, 0.05, np.inf, 0.05])
    got = _noalloc(_model(ffe.FFE_FP32C, U), N, 0.1, 0.0, h, T, d)
    assert np.isfinite(got[0]) and np.all(np.isnan(got[1:]))
    ref, _, _ = oracle.omega_batch(oracle.make_model(U=U), N, 0.1, 0.0, h[:1], T[:1], d[:1])
    assert abs(got[0] - ref[0]) / N**2 <= TOL[ffe.FFE_FP32C]


def test_noalloc_rejects_sizes_beyond_its_array():
    model = _model(ffe.FFE_FP32C, 2.0)
    dummy = ctypes.c_void_p(1)  # never dereferenced: the sizes are rejected first
    L = ffe.lib()
    assert L.ffe_omega_noalloc(ctypes.byref(model), 4096, 0.0, 0.0, dummy, dummy, dummy, 8, dummy,
                               None) == ffe.FFE_EINVAL
    assert L.ffe_omega_noalloc(ctypes.byref(model), 64, 0.0, 0.0, dummy, dummy, dummy, 513, dummy,
                               None) == ffe.FFE_EINVAL
