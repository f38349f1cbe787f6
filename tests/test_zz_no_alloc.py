"""ffe_omega_noalloc: Omega with every intermediate in the library's fixed
device array, for callers that cannot allocate device memory at call time
(a process whose free device memory belongs to its own pool, or a loop where
a cudaMalloc would synchronise the device).  Its results must equal those of
ffe_omega, the allocating entry point, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1412_8754_gb300 import ffe

pytestmark = pytest.mark.gpu

TOL = {ffe.FFE_FP64: 1e-9, ffe.FFE_FP32C: 2e-7}  # per lattice site, as for ffe_omega


def _noalloc(model, N, qx, qy, h, T, d):
    import torch

    dev = torch.device("cuda")
    th, tT, td = (torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev) for a in (h, T, d))
    out = torch.full((len(h),), float("nan"), dtype=torch.float64, device=dev)
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
    model = ffe.ffe_model(ffe.FFE_MODEL_RAGHU2, prec, -1.0, 1.3, -0.85, -0.85, 1.54, U, eta)
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


def test_noalloc_rejects_sizes_beyond_its_array():
    model = ffe.ffe_model(ffe.FFE_MODEL_RAGHU2, ffe.FFE_FP32C, -1.0, 1.3, -0.85, -0.85, 1.54, 2.0, 1.0)
    dummy = ctypes.c_void_p(1)  # never dereferenced: the sizes are rejected first
    L = ffe.lib()
    assert L.ffe_omega_noalloc(ctypes.byref(model), 4096, 0.0, 0.0, dummy, dummy, dummy, 8, dummy,
                               None) == ffe.FFE_EINVAL
    assert L.ffe_omega_noalloc(ctypes.byref(model), 64, 0.0, 0.0, dummy, dummy, dummy, 513, dummy,
                               None) == ffe.FFE_EINVAL
