"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (per lattice site, units of |t1|): FP64 1e-9, FP32+compensated 2e-7.
Argmin indices and phase labels must be identical to the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import search
from paper_1412_8754_gb300 import ffe, workloads

pytestmark = pytest.mark.gpu

TOL = {ffe.FFE_FP64: 1e-9, ffe.FFE_FP32C: 2e-7}
PRECS = [ffe.FFE_FP64, ffe.FFE_FP32C]


def per_site(a, b, N):
    return np.abs(np.asarray(a) - np.asarray(b)) / (np.asarray(N, dtype=float) ** 2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffe.lib()


@pytest.mark.parametrize("prec", PRECS)
def test_omega_random_points(prec):
    """Ragged lattices (N=8: 64 k-points; N=24: 576), both signs of q and h."""
    w = workloads.random_points(160, seed=11)
    U, eta = 2.5, 1.0
    m = oracle.make_model(U=U, eta_amp=eta)
    ref, _, _ = oracle.omega_batch(m, w["N"], w["qx"], w["qy"], w["h"], w["T"], w["delta"])
    with ffe.Context(prec=prec, U=U, eta_amp=eta) as ctx:
        got = ctx.omega(ffe.points(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["delta"]))
    err = per_site(got, ref, w["N"])
    assert err.max() <= TOL[prec], (err.max(), int(err.argmax()))


@pytest.mark.parametrize("prec", PRECS)
def test_omega_per_band(prec):
    """Omega_eps of the lower and upper band (each with its own Delta^2/U term) and their sum,
    ragged lattices, both signs of q and h."""
    w = workloads.random_points(120, seed=12)
    U = 3.0
    m = oracle.make_model(U=U)
    ref, ref_b, _ = oracle.omega_batch(m, w["N"], w["qx"], w["qy"], w["h"], w["T"], w["delta"], bands=True)
    pts = ffe.points(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["delta"])
    with ffe.Context(prec=prec, U=U) as ctx:
        got, got_b = ctx.omega(pts, bands=True)
        plain = ctx.omega(pts)
    for b in range(2):
        assert per_site(got_b[:, b], ref_b[:, b], w["N"]).max() <= TOL[prec], b
    assert per_site(got, ref, w["N"]).max() <= TOL[prec]
    assert per_site(got, plain, w["N"]).max() <= 2 * TOL[prec]


@pytest.mark.parametrize("N", [2, 4, 6, 10])
@pytest.mark.parametrize("prec", PRECS)
def test_omega_tiny_lattices(prec, N):
    m = oracle.make_model(U=2.0, eta_amp=4.0)
    d = np.linspace(0.0, 0.2, 7)
    ref, _, _ = oracle.omega_batch(m, N, 0.3, 0.1, 0.05, 0.01, d)
    with ffe.Context(prec=prec, U=2.0, eta_amp=4.0) as ctx:
        got = ctx.omega(ffe.points(N, 0.3, 0.1, 0.05, 0.01, d))
    assert per_site(got, ref, N).max() <= TOL[prec]


@pytest.mark.parametrize("U", [2.0, 4.0])
@pytest.mark.parametrize("prec", PRECS)
def test_small_bcs_grid(prec, U):
    """N=64, Q=0, h=0, T=0.005, 201 Delta in [0, 0.2]: Omega(Delta) and its argmin."""
    c = workloads.SMALL_BCS
    m = oracle.make_model(U=U)
    grid = np.linspace(c["lo"], c["hi"], c["n"])
    ref, _, _ = oracle.omega_batch(m, c["N"], 0.0, 0.0, 0.0, c["T"][0], grid)
    with ffe.Context(prec=prec, U=U) as ctx:
        res, om, eb = ctx.minimize(ffe.params(c["N"], 0.0, 0.0, 0.0, c["T"][0], c["lo"], c["hi"], c["n"]),
                                   want_grid=True)
    assert per_site(om, ref, c["N"]).max() <= TOL[prec]
    i = search.grid_argmin(ref)
    assert res["idx_star"][0] == i
    assert res["delta_star"][0] == grid[i]
    assert abs(res["omega_star"][0] - ref[i]) / c["N"] ** 2 <= TOL[prec]
    if U == 2.0:
        assert i == 0 and res["flags"][0] & ffe.FFE_FLAG_LOWER
    else:
        assert 100 < i < 130


def oracle_scan(m, N, qx, qy, h, T, grid):
    """Per (q, point) Omega grids, minima and labels, all from the oracle."""
    H, TT = np.meshgrid(h, T, indexing="ij")
    H, TT = H.ravel(), TT.ravel()
    npts = H.size
    Q = len(qx)
    qq = np.repeat(np.arange(Q), npts * len(grid))
    pp = np.tile(np.repeat(np.arange(npts), len(grid)), Q)
    dd = np.tile(grid, Q * npts)
    om, _, _ = oracle.omega_batch(m, N, np.asarray(qx)[qq], np.asarray(qy)[qq], H[pp], TT[pp], dd)
    om = om.reshape(Q, npts, len(grid))
    idx = np.array([[search.grid_argmin(om[q, p]) for p in range(npts)] for q in range(Q)])
    star = np.take_along_axis(om, idx[..., None], axis=2)[..., 0]
    labels, best = [], []
    for p in range(npts):
        lab, b = search.phase_label(star[:, p], om[:, p, 0],
                                    (np.asarray(qx) == 0) & (np.asarray(qy) == 0))
        labels.append(lab)
        best.append(b)
    return om, idx, star, np.array(labels), np.array(best)


def assert_same_scan(a, b):
    """Two executions of one scan agree bit for bit (the k-sum's order of addition is fixed)."""
    for name in a[0].dtype.names:
        assert np.array_equal(a[0][name], b[0][name], equal_nan=True), name
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("prec", PRECS)
def test_phase_scan_small(prec):
    """Grid phase scan: 6 q x (4 h x 2 T) x 41 Delta at N=32, U=4 (BCS and FF minima)."""
    N, U = 32, 4.0
    qx = np.array([0.0, 0.1, 0.2, 0.3, 0.45, 0.6])
    qy = np.zeros_like(qx)
    h = np.array([0.0, 0.05, 0.1, 0.15])
    T = np.array([0.004, 0.02])
    grid = np.linspace(0.0, 0.2, 41)
    m = oracle.make_model(U=U)
    om, idx, star, labels, best = oracle_scan(m, N, qx, qy, h, T, grid)
    with ffe.Context(prec=prec, U=U) as ctx:
        res, glab, gbest = ctx.phase_scan(N, qx, qy, h, T, n=41, lo=0.0, hi=0.2)
        again = ctx.phase_scan(N, qx, qy, h, T, n=41, lo=0.0, hi=0.2)  # the cached plan, refilled
    assert_same_scan((res, glab, gbest), again)
    assert np.array_equal(res["idx_star"], idx)
    assert per_site(res["omega_star"], star, N).max() <= TOL[prec]
    assert per_site(res["omega_lo"], om[..., 0], N).max() <= TOL[prec]
    assert np.array_equal(glab, labels), (glab, labels)
    assert np.array_equal(gbest, best)


def test_states_built_in_the_ksum_match_the_table(monkeypatch):
    """A plan too large for the FP32 k-state table builds the states inside the k-sum from the
    trig tables, with the same FP32 arithmetic: a scan gives the same bits either way."""
    N, U = 40, 4.0
    qx = np.array([0.0, 0.2, 0.45])
    args = (N, qx, np.zeros_like(qx), np.array([0.0, 0.05, 0.1]), np.array([0.004, 0.02]))
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        a = ctx.phase_scan(*args, n=33, lo=0.0, hi=0.2)
    monkeypatch.setenv("FFE_KSTATE_TABLE_MAX_BYTES", "0")
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        b = ctx.phase_scan(*args, n=33, lo=0.0, hi=0.2)
        plan = ctx.plan_phase_scan(*args, n=33, lo=0.0, hi=0.2)
        without = plan.stats()["device_bytes"]
        plan.destroy()
    monkeypatch.delenv("FFE_KSTATE_TABLE_MAX_BYTES")
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        plan = ctx.plan_phase_scan(*args, n=33, lo=0.0, hi=0.2)
        with_table = plan.stats()["device_bytes"]
        plan.destroy()
    assert_same_scan(a, b)
    assert with_table - without >= len(qx) * N * N * 20 - 20  # the table (20 B per (q, k)) was left out


@pytest.mark.parametrize("T, mixed", [(0.002, True), (0.6, False)])
def test_far_k_points_take_the_short_form(T, mixed):
    """FP32: a band far from the Fermi surface for every output of a work item (its log
    factors are 1 in FP32) is summed as W = c a; the others take the full term, with one
    exponential where c (R + |d|) >= 27 for every output. At low T most bands are far, at
    T = 0.6 none is (and none has one exponential); both match the oracle."""
    N, U = 48, 4.0
    qx = np.array([0.0, 0.3])
    qy = np.zeros_like(qx)
    h = np.linspace(0.0, 0.15, 8)
    Ts = np.array([T])
    grid = np.linspace(0.0, 0.2, 17)
    m = oracle.make_model(U=U)
    om, idx, star, labels, best = oracle_scan(m, N, qx, qy, h, Ts, grid)
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        plan = ctx.plan_phase_scan(N, qx, qy, h, Ts, n=17, lo=0.0, hi=0.2)
        plan.execute()
        res, lab, bq = plan.fetch()
        st = plan.stats()
        plan.destroy()
    frac = st["k_evals_near"] / (2 * st["k_evals"])  # full-term band evaluations, two bands per k-eval
    single = st["k_evals_single"] / (2 * st["k_evals"])
    closed = st["k_evals_far_closed"] / (2 * st["k_evals"])  # far bands that formed R and a
    if mixed:
        assert 0.0 < frac < 0.6, frac
        assert 0.0 < single <= frac, (single, frac)
        assert 0.0 <= closed <= 1.0 - frac, (closed, frac)
    else:
        assert frac == 1.0, frac
        assert single == 0.0 and closed == 0.0, (single, closed)
    assert np.array_equal(res["idx_star"], idx)
    assert per_site(res["omega_star"], star, N).max() <= TOL[ffe.FFE_FP32C]
    assert per_site(res["omega_lo"], om[..., 0], N).max() <= TOL[ffe.FFE_FP32C]
    assert np.array_equal(lab, labels) and np.array_equal(bq, best)


def test_fp32c_error_bound_covers_fp64():
    """Every FP32+compensated value lies within its stated bound of the FP64 kernel's."""
    w = workloads.uneven_jobs(24, seed=5, sizes=(16, 32, 48, 64))
    ps = ffe.params(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["lo"], w["hi"], w["n"])
    with ffe.Context(prec=ffe.FFE_FP64, U=3.0) as c64, ffe.Context(prec=ffe.FFE_FP32C, U=3.0) as c32:
        r64, g64, e64 = c64.minimize(ps, want_grid=True)
        r32, g32, e32 = c32.minimize(ps, want_grid=True)
    assert np.all(e64 == 0)
    assert np.all(np.abs(g32 - g64) <= e32 + 1e-12 * np.abs(g64))
    assert np.array_equal(r32["idx_star"], r64["idx_star"])


def test_uneven_jobs_small_vs_oracle():
    """Uneven lattices and grid lengths in one launch (shape of the 512-job batch, small N)."""
    w = workloads.uneven_jobs(12, seed=3, sizes=(8, 16, 24, 40))
    w["n"] = np.minimum(w["n"], 60)
    m = oracle.make_model(U=3.0)
    ps = ffe.params(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["lo"], w["hi"], w["n"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=3.0) as ctx:
        res, grid, _ = ctx.minimize(ps, want_grid=True)
    off = 0
    for j in range(len(ps)):
        n = int(w["n"][j])
        g = np.linspace(0.0, 0.2, n)
        ref, _, _ = oracle.omega_batch(m, int(w["N"][j]), w["qx"][j], 0.0, w["h"][j], w["T"][j], g)
        assert per_site(grid[off:off + n], ref, w["N"][j]).max() <= TOL[ffe.FFE_FP32C]
        assert res["idx_star"][j] == search.grid_argmin(ref)
        off += n


def test_plan_replay_is_deterministic():
    N = 64
    qx = np.array([0.0, 0.2, 0.4])
    with ffe.Context(prec=ffe.FFE_FP32C, U=4.0) as ctx:
        plan = ctx.plan_phase_scan(N, qx, np.zeros(3), np.array([0.0, 0.06]), np.array([0.005]), n=64)
        plan.execute()
        a = plan.fetch()
        plan.execute()
        plan.execute()
        b = plan.fetch()
        ms, cnt = plan.kernel_ms()
        info = plan.stats()
        plan.destroy()
    assert a[0].tobytes() == b[0].tobytes()
    assert np.array_equal(a[1], b[1])
    assert cnt == 3 and ms > 0
    assert info["k_evals"] == N * N * 3 * 2 * 64 and info["launches"] >= 4


def test_invalid_arguments_are_rejected_before_launch():
    with ffe.Context(prec=ffe.FFE_FP32C) as ctx:
        for bad in (ffe.points(7, 0, 0, 0, 0.01, 0.1), ffe.points(16, 0, 0, 0, 0.0, 0.1),
                    ffe.points(16, 0, 0, 0, float("nan"), 0.1), ffe.points(9000, 0, 0, 0, 0.1, 0.1)):
            with pytest.raises(ffe.FFEError) as e:
                ctx.omega(bad)
            assert e.value.status == ffe.FFE_EINVAL
        with pytest.raises(ffe.FFEError):
            ctx.minimize(ffe.params(16, 0, 0, 0, 0.01, 0.2, 0.1, 10))  # lo > hi
        with pytest.raises(ffe.FFEError):
            ctx.phase_scan(16, [0.1], [0.0], [0.0], [0.01], n=8)  # no q = 0
        # the context stays usable
        ok = ctx.omega(ffe.points(16, 0, 0, 0, 0.01, 0.1))
        assert np.isfinite(ok[0])


def oracle_golden(m, N, qx, qy, h, T, lo, hi, steps):
    """Lockstep golden-section of the oracle over many points (broadcast arrays)."""
    qx, qy, h, T = np.broadcast_arrays(np.asarray(qx, float), np.asarray(qy, float),
                                       np.asarray(h, float), np.asarray(T, float))

    def ev(d):
        om, _, _ = oracle.omega_batch(m, N, qx.ravel(), qy.ravel(), h.ravel(), T.ravel(), d)
        return om

    n = qx.size
    return search.golden_section_batch(ev, np.full(n, lo), np.full(n, hi), steps)


@pytest.mark.parametrize("prec", PRECS)
def test_minimize_bands_grid_vs_oracle(prec):
    """Per-band independent minimisation on a grid: each band's argmin of its own Omega_eps is
    the oracle's, index for index."""
    U, n = 4.0, 41
    rng = np.random.default_rng(23)
    k = 16
    N = rng.choice(np.array([16, 24, 32]), size=k).astype(np.int32)
    qx = rng.uniform(0, 0.5, k)
    qx[:3] = 0.0
    h = rng.uniform(0, 0.12, k)
    T = rng.uniform(0.002, 0.03, k)
    m = oracle.make_model(U=U)
    grid = np.linspace(0.0, 0.2, n)
    with ffe.Context(prec=prec, U=U) as ctx:
        res = ctx.minimize_bands(ffe.params(N, qx, 0.0, h, T, 0.0, 0.2, n))
    assert res.shape == (k, 2)
    interior = 0
    for i in range(k):
        _, ob, _ = oracle.omega_batch(m, int(N[i]), qx[i], 0.0, h[i], T[i], grid, bands=True)
        for b in range(2):
            idx = search.grid_argmin(ob[:, b])
            interior += 0 < idx < n - 1
            assert res[i, b]["idx_star"] == idx, (i, b, res[i, b]["idx_star"], idx)
            assert per_site(res[i, b]["omega_star"], ob[idx, b], N[i]) <= TOL[prec]
            assert per_site(res[i, b]["omega_lo"], ob[0, b], N[i]) <= TOL[prec]
    assert interior > 0  # some band has a gap of its own


@pytest.mark.parametrize("prec", PRECS)
def test_minimize_bands_golden_vs_oracle(prec):
    """Per-band golden-section searches against the oracle's on each band's Omega_eps."""
    N, U, steps = 24, 4.0, 20
    rng = np.random.default_rng(29)
    k = 12
    qx = rng.uniform(0, 0.4, k)
    h = rng.uniform(0, 0.1, k)
    T = rng.uniform(0.002, 0.02, k)
    m = oracle.make_model(U=U)
    with ffe.Context(prec=prec, U=U) as ctx:
        res = ctx.minimize_bands(ffe.params(N, qx, 0.0, h, T, 0.0, 0.2, steps), search=ffe.FFE_SEARCH_GOLDEN)
    for b in range(2):
        def ev(d, b=b):
            _, ob, _ = oracle.omega_batch(m, N, qx, 0.0, h, T, d, bands=True)
            return ob[:, b]

        xb, fb, f0 = search.golden_section_batch(ev, np.zeros(k), np.full(k, 0.2), steps)
        assert per_site(res[:, b]["omega_lo"], f0, N).max() <= TOL[prec]
        at_gpu = ev(res[:, b]["delta_star"])
        assert per_site(res[:, b]["omega_star"], at_gpu, N).max() <= TOL[prec]
        slack = {ffe.FFE_FP64: 1e-11, ffe.FFE_FP32C: 1e-9}[prec]
        assert np.all((at_gpu - fb) / N**2 <= slack)
        assert np.array_equal(res[:, b]["flags"] & ffe.FFE_FLAG_LOWER != 0, xb == 0.0)


@pytest.mark.parametrize("prec", PRECS)
def test_golden_phase_scan_vs_oracle(prec):
    """Golden phase scan: 5 q x (3 h x 2 T) at N=32, U=4; labels equal to the oracle's."""
    N, U, steps = 32, 4.0, 20
    qx = np.array([0.0, 0.15, 0.3, 0.45, 0.6])
    h = np.array([0.0, 0.07, 0.14])
    T = np.array([0.003, 0.02])
    m = oracle.make_model(U=U)
    H, TT = np.meshgrid(h, T, indexing="ij")
    Q = np.repeat(qx, H.size)
    HH = np.tile(H.ravel(), len(qx))
    TTT = np.tile(TT.ravel(), len(qx))
    xb, fb, f0 = oracle_golden(m, N, Q, 0.0, HH, TTT, 0.0, 0.2, steps)
    xb, fb, f0 = (a.reshape(len(qx), H.size) for a in (xb, fb, f0))
    labels, best = [], []
    for p in range(H.size):
        lab, b = search.phase_label(fb[:, p], f0[:, p], qx == 0.0)
        labels.append(lab)
        best.append(b)
    with ffe.Context(prec=prec, U=U) as ctx:
        res, glab, gbest = ctx.phase_scan(N, qx, np.zeros_like(qx), h, T, search=ffe.FFE_SEARCH_GOLDEN,
                                          n=steps, lo=0.0, hi=0.2)
    assert per_site(res["omega_lo"], f0, N).max() <= TOL[prec]
    assert per_site(res["omega_star"], fb, N).max() <= TOL[prec] + 1e-9
    assert np.array_equal(glab, np.array(labels)), (glab, labels)
    assert np.array_equal(gbest, np.array(best))
    assert np.all(res["idx_star"] == -1)


def test_golden_plan_replay():
    N = 32
    qx = np.array([0.0, 0.3])
    with ffe.Context(prec=ffe.FFE_FP32C, U=4.0) as ctx:
        plan = ctx.plan_phase_scan(N, qx, np.zeros(2), np.array([0.0, 0.1]), np.array([0.004]),
                                   search=ffe.FFE_SEARCH_GOLDEN, n=12)
        plan.execute()
        a = plan.fetch()
        plan.execute()
        b = plan.fetch()
        info = plan.stats()
        plan.destroy()
    assert a[0].tobytes() == b[0].tobytes()
    assert info["k_evals"] == N * N * 2 * 2 * (3 + 12)  # every line evaluated 3 + steps times


def test_uneven_batch_full_size_sampled():
    """512 jobs, N in {256, 512, 1024, 2048}, 32..256 Delta each, one graph-captured
    persistent launch (the plan the benchmark times).  Sampled jobs are checked
    against the oracle at the argmin, its neighbours and Delta = 0."""
    w = workloads.uneven_jobs(512, seed=1234)
    U = 2.0
    ps = ffe.params(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["lo"], w["hi"], w["n"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        plan = ctx.plan_minimize(ps)
        plan.execute()
        res, grid, err = plan.fetch_minimize(want_grid=True)
        info = plan.stats()
        plan.destroy()
    assert info["k_evals"] == float(np.sum(w["N"].astype(float) ** 2 * w["n"]))
    m = oracle.make_model(U=U)
    offs = np.concatenate([[0], np.cumsum(w["n"])[:-1]])
    rng = np.random.default_rng(99)
    pick = rng.choice(512, 6, replace=False)
    rows = []
    for j in pick:
        n = int(w["n"][j])
        g = np.linspace(0.0, 0.2, n)
        i = int(res["idx_star"][j])
        for ii in sorted({0, max(i - 1, 0), i, min(i + 1, n - 1)}):
            rows.append((j, ii, g[ii]))
    J = np.array([r[0] for r in rows])
    ref, _, _ = oracle.omega_batch(m, w["N"][J], w["qx"][J], 0.0, w["h"][J], w["T"][J], [r[2] for r in rows])
    got = np.array([grid[offs[r[0]] + r[1]] for r in rows])
    assert per_site(got, ref, w["N"][J]).max() <= TOL[ffe.FFE_FP32C]
    for j in pick:  # the GPU argmin is a local minimum of the oracle's Omega
        sel = [k for k, r in enumerate(rows) if r[0] == j]
        vals = {rows[k][1]: ref[k] for k in sel}
        i = int(res["idx_star"][j])
        assert all(vals[i] <= v + 1e-12 * abs(v) for v in vals.values())
    assert np.all(np.abs(grid) > 0) and np.all(err >= 0)


def test_fflo_scan_full_size_sampled():
    """The benchmark's FFLO scan at full size (N = 1024, 64 q x 32 h x 256 Delta, one T, U = 2)
    in the plan and launch configuration the benchmark times.  For two h values and every q the
    oracle evaluates Omega at the GPU argmin, its neighbours and Delta = 0: values per site
    within the FP32C tolerance, the argmin a local minimum of the oracle's Omega, and the label
    and best q those the oracle's values give."""
    cfg = workloads.fflo_scan()
    U, N, T = 2.0, cfg["N"], float(cfg["T"][0])
    grid = np.linspace(cfg["lo"], cfg["hi"], cfg["n"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        plan = ctx.plan_phase_scan(N, cfg["qx"], cfg["qy"], cfg["h"], cfg["T"], n=cfg["n"], lo=cfg["lo"],
                                   hi=cfg["hi"])
        plan.execute()
        res, labels, best = plan.fetch()
        plan.destroy()
    m = oracle.make_model(U=U)
    nq = len(cfg["qx"])
    for ih in (3, 27):  # one point per (h, T): index ih of the h list
        rows = []
        for q in range(nq):
            i = int(res["idx_star"][q, ih])
            for ii in sorted({0, max(i - 1, 0), i, min(i + 1, cfg["n"] - 1)}):
                rows.append((q, ii))
        Q = np.array([r[0] for r in rows])
        ref, _, _ = oracle.omega_batch(m, N, cfg["qx"][Q], 0.0, cfg["h"][ih], T, grid[[r[1] for r in rows]])
        val = {r: ref[k] for k, r in enumerate(rows)}
        star = np.array([val[(q, int(res["idx_star"][q, ih]))] for q in range(nq)])
        zero = np.array([val[(q, 0)] for q in range(nq)])
        assert per_site(res["omega_star"][:, ih], star, N).max() <= TOL[ffe.FFE_FP32C]
        assert per_site(res["omega_lo"][:, ih], zero, N).max() <= TOL[ffe.FFE_FP32C]
        for q in range(nq):
            i = int(res["idx_star"][q, ih])
            assert all(val[(q, i)] <= v + 1e-12 * abs(v) for (qq, _), v in val.items() if qq == q)
        want, wq = search.phase_label(star, zero, cfg["qx"] == 0.0)
        assert labels[ih] == want and best[ih] == wq


def test_golden_phase_diagram_full_size_sampled():
    """The phase diagram's golden-section search at its full lattice (N = 2048, 24 reductions on
    [0, 0.2]) on a few (q, h, T) lines: Omega at the GPU's Delta* and at Delta = 0 per site within
    the FP32C tolerance, and Delta* no worse than the oracle at Delta* -+ 2e-3 (a minimum of the
    oracle's Omega up to the FP32C tolerance)."""
    pd = workloads.phase_diagram()
    U, N = 2.0, pd["N"]
    qx = pd["qx"][[0, 21, 42]]
    h, T = pd["h"][[0, 40]], pd["T"][[0, 20]]
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        res, labels, best = ctx.phase_scan(N, qx, np.zeros_like(qx), h, T, search=ffe.FFE_SEARCH_GOLDEN,
                                           n=pd["n"], lo=pd["lo"], hi=pd["hi"])
    m = oracle.make_model(U=U)
    pts = [(q, ih, it) for q in range(len(qx)) for ih in range(len(h)) for it in range(len(T))]
    d = np.array([res["delta_star"][q, ih * len(T) + it] for q, ih, it in pts])
    args = [(q, ih, it, x) for (q, ih, it), ds in zip(pts, d) for x in (ds, 0.0, max(ds - 2e-3, 0.0), ds + 2e-3)]
    ref, _, _ = oracle.omega_batch(m, N, qx[[a[0] for a in args]], 0.0, h[[a[1] for a in args]],
                                   T[[a[2] for a in args]], [a[3] for a in args])
    ref = ref.reshape(len(pts), 4)
    for k, (q, ih, it) in enumerate(pts):
        pt = ih * len(T) + it
        assert per_site(res["omega_star"][q, pt], ref[k, 0], N) <= TOL[ffe.FFE_FP32C]
        assert per_site(res["omega_lo"][q, pt], ref[k, 1], N) <= TOL[ffe.FFE_FP32C]
        assert (ref[k, 0] - ref[k, 2:].min()) / N ** 2 <= TOL[ffe.FFE_FP32C]


def test_autotune_keeps_results():
    w = workloads.uneven_jobs(40, seed=8, sizes=(64, 128, 256))
    ps = ffe.params(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["lo"], w["hi"], w["n"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=3.0) as ctx:
        plan = ctx.plan_minimize(ps)
        plan.execute()
        a, ga, _ = plan.fetch_minimize(want_grid=True)
        shape = plan.autotune()
        plan.execute()
        b, gb, _ = plan.fetch_minimize(want_grid=True)
        plan.destroy()
    assert shape["kpt"] in (2, 4, 8) and shape["block"] in (128, 256)
    assert np.array_equal(a["idx_star"], b["idx_star"])
    assert per_site(ga, gb, np.repeat(w["N"], w["n"])).max() <= 1e-8


@pytest.mark.parametrize("prec", PRECS)
def test_per_band_coupling(prec):
    """Each band with its own coupling U_eps (U_band = (9, 3)): Omega and Omega_eps at random points,
    and the per-band grid minimisation at Q = 0 and small q, h against the oracle, index for index;
    the two bands' minima differ."""
    Ub = (9.0, 3.0)
    w = workloads.random_points(60, seed=31)
    m = oracle.make_model(U=4.0, U_band=Ub)
    ref, ref_b, _ = oracle.omega_batch(m, w["N"], w["qx"], w["qy"], w["h"], w["T"], w["delta"], bands=True)
    n, N = 41, 32
    qx = np.array([0.0, 0.0, 0.1, 0.2])
    h = np.array([0.0, 0.02, 0.01, 0.03])
    T = np.array([0.003, 0.005, 0.004, 0.002])
    grid = np.linspace(0.0, 0.3, n)
    with ffe.Context(prec=prec, U=4.0, U_band=Ub) as ctx:
        got, got_b = ctx.omega(ffe.points(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["delta"]), bands=True)
        res = ctx.minimize_bands(ffe.params(N, qx, 0.0, h, T, 0.0, 0.3, n))
    assert per_site(got, ref, w["N"]).max() <= TOL[prec]
    for b in range(2):
        assert per_site(got_b[:, b], ref_b[:, b], w["N"]).max() <= TOL[prec]
    differ = 0
    for i in range(len(qx)):
        _, ob, _ = oracle.omega_batch(m, N, qx[i], 0.0, h[i], T[i], grid, bands=True)
        idx = [search.grid_argmin(ob[:, b]) for b in range(2)]
        for b in range(2):
            assert res[i, b]["idx_star"] == idx[b], (i, b, res[i, b]["idx_star"], idx[b])
            assert per_site(res[i, b]["omega_star"], ob[idx[b], b], N) <= TOL[prec]
        differ += idx[0] != idx[1] and min(idx) > 0
    assert differ >= 2
