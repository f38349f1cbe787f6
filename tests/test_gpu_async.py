"""Stream-ordered entry points (device arrays in and out, no host synchronisation) against the
host-buffer calls and the oracle, and cached plans refilled with new values of the same shape."""
import numpy as np
import pytest

import oracle
from oracle import search
from paper_1412_8754_gb300 import ffe, workloads

from test_gpu_parity import PRECS, TOL, per_site

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    return t


def dev(torch, a, dtype=None):
    return torch.as_tensor(np.asarray(a, dtype=dtype or np.float64), device="cuda")


@pytest.mark.parametrize("prec", PRECS)
def test_omega_async_matches_oracle_and_host_call(prec, torch):
    """Ragged batch (77 points, N = 24) on a side stream, per band and total; an invalid point is NaN."""
    rng = np.random.default_rng(41)
    U, N, qx, qy, n = 4.0, 24, 0.27, 0.05, 77
    h = rng.uniform(-0.12, 0.12, n)
    T = np.where(np.arange(n) % 3 == 0, 0.002, rng.uniform(0.004, 0.04, n))
    d = rng.uniform(0.0, 0.2, n)
    ref, ref_b, _ = oracle.omega_batch(oracle.make_model(U=U), N, qx, qy, h, T, d, bands=True)
    T_bad = T.copy()
    T_bad[5] = 0.0
    side = torch.cuda.Stream()
    with ffe.Context(prec=prec, U=U) as ctx:
        host = ctx.omega(ffe.points(N, qx, qy, h, T, d))
        th, tT, td = dev(torch, h), dev(torch, T_bad), dev(torch, d)
        om = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
        ob = torch.full((n, 2), 7.0, dtype=torch.float64, device="cuda")
        om2 = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ffe.ffe_omega_async(ctx.handle, N, qx, qy, th, tT, td, om, ob, stream=side)
            ffe.ffe_omega_async(ctx.handle, N, qx, qy, th, dev(torch, T), td, om2, stream=side)
        side.synchronize()
        got, got_b, got2 = om.cpu().numpy(), ob.cpu().numpy(), om2.cpu().numpy()
    ok = np.arange(n) != 5
    assert np.isnan(got[5]) and np.all(np.isnan(got_b[5]))
    assert per_site(got[ok], ref[ok], N).max() <= TOL[prec]
    for b in range(2):
        assert per_site(got_b[ok, b], ref_b[ok, b], N).max() <= TOL[prec]
    assert per_site(got2, ref, N).max() <= TOL[prec]
    assert per_site(got2, host, N).max() <= 2 * TOL[prec]


def test_omega_async_three_band(torch):
    from oracle import threeband

    rng = np.random.default_rng(42)
    N, U, n = 16, 1.2, 40
    h = rng.uniform(0.0, 0.02, n)
    T = rng.uniform(0.001, 0.004, n)
    d = rng.uniform(0.0, 0.05, n)
    ref, ref_b, _ = threeband.omega_batch(N, 0.1, 0.0, h, T, d, U=U, bands=True)
    with ffe.Context(prec=ffe.FFE_FP64, U=U, model="daghofer3") as ctx:
        om = torch.zeros(n, dtype=torch.float64, device="cuda")
        ob = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        ffe.ffe_omega_async(ctx.handle, N, 0.1, 0.0, dev(torch, h), dev(torch, T), dev(torch, d), om, ob)
        torch.cuda.synchronize()
    tol = TOL[ffe.FFE_FP64] * 0.08  # |t1| = 0.08 eV in the three-band model
    assert per_site(om.cpu().numpy(), ref, N).max() <= tol
    assert per_site(ob.cpu().numpy(), ref_b, N).max() <= tol


@pytest.mark.parametrize("search_kind", [ffe.FFE_SEARCH_GRID, ffe.FFE_SEARCH_GOLDEN])
def test_minimize_async_matches_host_call_and_refills(search_kind, torch):
    """Two calls of one shape with different (h, T) (the second refills the cached plan, its work
    items' far windows included): the device results equal the host-buffer call's, bit for bit,
    and the grid argmins are the oracle's."""
    U, n_pts = 4.0, 12
    rng = np.random.default_rng(43)
    N = rng.choice(np.array([16, 24, 32]), size=n_pts).astype(np.int32)
    qx = rng.uniform(0.0, 0.4, n_pts)
    steps = 33 if search_kind == ffe.FFE_SEARCH_GRID else 16
    m = oracle.make_model(U=U)
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        for call, (hmax, Tlo, Thi) in enumerate(((0.05, 0.002, 0.004), (0.12, 0.01, 0.03))):
            h = rng.uniform(0.0, hmax, n_pts)
            T = rng.uniform(Tlo, Thi, n_pts)
            ps = ffe.params(N, qx, 0.0, h, T, 0.0, 0.2, steps)
            buf = ffe.result_buffer(n_pts)
            grid = torch.zeros(int(ps["n"].sum()), dtype=torch.float64, device="cuda") \
                if search_kind == ffe.FFE_SEARCH_GRID else None
            ffe.ffe_minimize_async(ctx.handle, ps, buf, search=search_kind, omega_grid=grid)
            torch.cuda.synchronize()
            got = ffe.as_results(buf)
            if search_kind == ffe.FFE_SEARCH_GRID:
                want, wgrid, _ = ctx.minimize(ps, want_grid=True)
                assert np.array_equal(grid.cpu().numpy(), wgrid)
                for i in range(n_pts):
                    ref, _, _ = oracle.omega_batch(m, int(N[i]), qx[i], 0.0, h[i], T[i], np.linspace(0, 0.2, steps))
                    assert got["idx_star"][i] == search.grid_argmin(ref), (call, i)
            else:
                want = ctx.minimize(ps, search=search_kind)
            for name in ("delta_star", "omega_star", "omega_lo", "idx_star", "flags"):
                assert np.array_equal(got[name], want[name]), (call, name)
            assert np.all((got["flags"] & ffe.FFE_FLAG_INVALID) == 0)


@pytest.mark.parametrize("prec", PRECS)
def test_phase_scan_async_matches_host_call(prec, torch):
    c = workloads.ff_scan(n_q=11, n_h=6)
    with ffe.Context(prec=prec, **workloads.FF_MODEL) as ctx:
        want = ctx.phase_scan(c["N"], c["qx"], c["qy"], c["h"], c["T"], n=c["n"], lo=c["lo"], hi=c["hi"])
        npts = len(c["h"]) * len(c["T"])
        buf = ffe.result_buffer(len(c["qx"]) * npts)
        lab = torch.full((npts,), -1, dtype=torch.int8, device="cuda")
        best = torch.full((npts,), -7, dtype=torch.int32, device="cuda")
        for _ in range(2):  # the second call refills the cached plan
            ffe.ffe_phase_scan_async(ctx.handle, c["N"], c["qx"], c["qy"], c["h"], c["T"], buf, lab, best, n=c["n"],
                                     lo=c["lo"], hi=c["hi"], stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
    got = ffe.as_results(buf).reshape(len(c["qx"]), npts)
    for name in ("delta_star", "omega_star", "idx_star"):
        assert np.array_equal(got[name], want[0][name]), name
    assert np.array_equal(lab.cpu().numpy(), want[1]) and np.array_equal(best.cpu().numpy(), want[2])
    assert (want[1] == search.FFLO).any()


def test_cached_scan_plan_refilled_with_new_temperatures():
    """ffe_phase_scan reuses its plan for a scan of the same shape; the work items' far windows
    (which depend on T_max and the h range) are rebuilt, so a scan at higher T gives what a fresh
    context gives."""
    N, U = 32, 4.0
    qx = np.array([0.0, 0.2, 0.4])
    h = np.array([0.0, 0.05, 0.1])
    args = dict(n=33, lo=0.0, hi=0.2)
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        ctx.phase_scan(N, qx, np.zeros(3), h, np.array([0.002]), **args)
        again = ctx.phase_scan(N, qx, np.zeros(3), h + 0.01, np.array([0.03]), **args)
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as fresh:
        ref = fresh.phase_scan(N, qx, np.zeros(3), h + 0.01, np.array([0.03]), **args)
    for name in ("delta_star", "omega_star", "omega_lo", "idx_star"):
        assert np.array_equal(again[0][name], ref[0][name]), name
    assert np.array_equal(again[1], ref[1]) and np.array_equal(again[2], ref[2])


@pytest.mark.parametrize("kind", [ffe.FFE_SEARCH_GRID, ffe.FFE_SEARCH_GOLDEN])
def test_refilled_plan_with_new_values_equals_a_fresh_plan(kind):
    """A cached scan plan refilled with other q, h, T values and another Delta range (same
    shapes: the work items keep their structure and only their windows are recomputed) gives
    the same bits as a plan built for those values from scratch; many h blocks, so many
    segments with different windows."""
    N, U = 64, 4.0
    n = 48 if kind == ffe.FFE_SEARCH_GRID else 12
    first = dict(qx=np.linspace(0.0, 0.5, 5), h=np.linspace(0.0, 0.12, 40), T=np.array([0.002, 0.01]), lo=0.0,
                 hi=0.2)
    second = dict(qx=np.linspace(0.0, 0.3, 5), h=np.linspace(0.02, 0.2, 40), T=np.array([0.004, 0.03]), lo=0.0,
                  hi=0.3)
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        for v in (first, second):
            again = ctx.phase_scan(N, v["qx"], np.zeros(5), v["h"], v["T"], search=kind, n=n, lo=v["lo"],
                                   hi=v["hi"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as fresh:
        v = second
        ref = fresh.phase_scan(N, v["qx"], np.zeros(5), v["h"], v["T"], search=kind, n=n, lo=v["lo"], hi=v["hi"])
    for name in ("delta_star", "omega_star", "omega_lo", "idx_star", "flags"):
        assert np.array_equal(again[0][name], ref[0][name]), name
    assert np.array_equal(again[1], ref[1]) and np.array_equal(again[2], ref[2])
