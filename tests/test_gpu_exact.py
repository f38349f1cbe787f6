"""Discrete outputs of the CUDA path against the oracle, exactly: argmin indices, golden-section
Delta*, phase labels and best q (Alg. 1), on scans that reach every label -- normal, BCS and FF --
and on whole Delta grids of full-size (N = 1024) lines on both sides of a first-order transition.

Values per site within the tolerances of the parity tests (FP64 1e-9, FP32+compensated 2e-7, units
of |t1|); indices and labels identical.  A golden-section search must take the oracle's decisions
wherever the oracle's own comparisons are decided by more than four times the per-value tolerance
(then any evaluation within the tolerance takes the same decisions): its Delta* is the oracle's, or,
past the first comparison inside that band, lies in the bracket the oracle had there; every Delta*
reaches the oracle's minimum within the tolerance.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import search
from paper_1412_8754_gb300 import ffe, qgrid, workloads

from test_gpu_parity import PRECS, TOL, oracle_scan, per_site

pytestmark = pytest.mark.gpu


def ff_context(prec):
    return ffe.Context(prec=prec, **workloads.FF_MODEL)


def ff_oracle_model():
    return oracle.make_model(**workloads.FF_MODEL)


@pytest.fixture(scope="module")
def ff_oracle():
    """Oracle grids, argmins and labels of the FF scan (N = 64)."""
    c = workloads.ff_scan()
    grid = np.linspace(c["lo"], c["hi"], c["n"])
    return oracle_scan(ff_oracle_model(), c["N"], c["qx"], c["qy"], c["h"], c["T"], grid)


@pytest.mark.parametrize("prec", PRECS)
def test_ff_grid_scan_is_exact(prec, ff_oracle):
    """mu = 3.8, U = 5: the grid scan reaches normal, BCS and FF points; every argmin index, label
    and best q is the oracle's."""
    c = workloads.ff_scan()
    om, idx, star, labels, best = ff_oracle
    assert (labels == search.FFLO).sum() >= 3 and (labels == search.BCS).sum() >= 3
    assert (labels == search.NORMAL).sum() >= 3
    with ff_context(prec) as ctx:
        res, glab, gbest = ctx.phase_scan(c["N"], c["qx"], c["qy"], c["h"], c["T"], n=c["n"], lo=c["lo"],
                                          hi=c["hi"])
    assert np.array_equal(res["idx_star"], idx)
    assert per_site(res["omega_star"], star, c["N"]).max() <= TOL[prec]
    assert per_site(res["omega_lo"], om[..., 0], c["N"]).max() <= TOL[prec]
    assert np.array_equal(glab, labels), (glab, labels)
    assert np.array_equal(gbest, best), (gbest, best)
    ff = labels == search.FFLO
    assert np.all(c["qx"][gbest[ff]] > 0)


def golden_exactness(m, N, qx, qy, h, T, lo, hi, steps, res, prec):
    """Checks every line's golden-section outcome against the oracle's own search.

    The oracle records its brackets and the margin |Omega(x1) - Omega(x2)| of each decision.  Up to
    the first decision whose margin is within four times the per-value tolerance, the GPU (whose
    values lie within the tolerance of the oracle's) must take the same decisions on the same
    points: its Delta* is then one of the points the oracle evaluated before that decision, or
    lies inside the bracket that decision splits.  A line with no such decision evaluates the
    oracle's points exactly, and its Delta* is the oracle's unless the two lowest values are
    within the band too.  Returns (lines with Delta* identical, xb, fb, f0)."""
    qx, qy, h, T = (np.asarray(a, float).ravel() for a in np.broadcast_arrays(qx, qy, h, T))

    def ev(d):
        return oracle.omega_batch(m, N, qx, qy, h, T, d)[0]

    n = qx.size
    xb, fb, f0, tr = search.golden_section_batch(ev, np.full(n, lo), np.full(n, hi), steps, trace=True)
    thr = 4.0 * TOL[prec] * N * N
    d_gpu = res["delta_star"].ravel()
    close = tr["margin"] <= thr
    first = np.where(close.any(axis=0), close.argmax(axis=0), steps)
    fs = np.sort(tr["f"], axis=0)
    for i in range(n):
        k = int(first[i])
        seen = tr["x"][:3 + k, i]
        if k == steps:
            assert d_gpu[i] in seen, (i, d_gpu[i])
            if fs[1, i] - fs[0, i] > thr:
                assert d_gpu[i] == xb[i], (i, d_gpu[i], xb[i])
        else:
            assert d_gpu[i] in seen or tr["a"][k, i] <= d_gpu[i] <= tr["b"][k, i], (i, k, d_gpu[i])
    assert per_site(res["omega_lo"].ravel(), f0, N).max() <= TOL[prec]
    # every line: the GPU's Delta* is a point whose oracle value is the oracle's minimum up to
    # the tolerance, and the GPU's value there agrees with the oracle's
    at_gpu = ev(d_gpu)
    assert per_site(res["omega_star"].ravel(), at_gpu, N).max() <= TOL[prec]
    assert np.all((at_gpu - fb) / N**2 <= 2.0 * TOL[prec])
    return int(np.sum(d_gpu == xb)), xb, fb, f0


@pytest.mark.parametrize("prec", PRECS)
def test_golden_minimize_is_exact(prec):
    """40 random lines at N = 32, U = 4, 24 reductions on [0, 0.2]."""
    N, U, steps = 32, 4.0, 24
    rng = np.random.default_rng(17)
    n = 40
    qx = rng.uniform(0, 0.5, n)
    qx[:4] = 0.0
    h = rng.uniform(0, 0.12, n)
    T = rng.uniform(0.002, 0.03, n)
    with ffe.Context(prec=prec, U=U) as ctx:
        res = ctx.minimize(ffe.params(N, qx, 0.0, h, T, 0.0, 0.2, steps), search=ffe.FFE_SEARCH_GOLDEN)
    same, xb, _, _ = golden_exactness(oracle.make_model(U=U), N, qx, 0.0, h, T, 0.0, 0.2, steps, res, prec)
    print(f"golden lines with Delta* identical to the oracle's: {same} of {n}")
    assert np.array_equal(res["flags"] & ffe.FFE_FLAG_LOWER != 0, res["delta_star"] == 0.0)


@pytest.mark.parametrize("prec", PRECS)
def test_ff_golden_scan_is_exact(prec):
    """The FF scan with 20 golden-section reductions: Delta* per line (outside the tolerance band),
    labels and best q from the oracle's own golden search."""
    c = workloads.ff_scan()
    steps = 20
    N = c["N"]
    H, TT = np.meshgrid(c["h"], c["T"], indexing="ij")
    npts = H.size
    Q = np.repeat(c["qx"], npts)
    with ff_context(prec) as ctx:
        res, glab, gbest = ctx.phase_scan(N, c["qx"], c["qy"], c["h"], c["T"], search=ffe.FFE_SEARCH_GOLDEN,
                                          n=steps, lo=c["lo"], hi=c["hi"])
    same, xb, fb, f0 = golden_exactness(ff_oracle_model(), N, Q, 0.0, np.tile(H.ravel(), len(c["qx"])),
                                        np.tile(TT.ravel(), len(c["qx"])), c["lo"], c["hi"], steps, res, prec)
    fb, f0 = fb.reshape(len(c["qx"]), npts), f0.reshape(len(c["qx"]), npts)
    labels, best = zip(*(search.phase_label(fb[:, p], f0[:, p], c["qx"] == 0.0) for p in range(npts)))
    labels, best = np.array(labels), np.array(best)
    print(f"FF golden lines with Delta* identical to the oracle's: {same} of {fb.size}")
    assert (labels == search.FFLO).sum() >= 3
    assert np.array_equal(glab, labels), (glab, labels)
    assert np.array_equal(gbest, best), (gbest, best)


def ff_surrogate(ctx, N, seed):
    """A surrogate trained on the FF model's own free energies (library k-sum at N) over the box of
    the FF scan: q in [0, 0.32], h in [0.025, 0.055], T in [0.0015, 0.0035], Delta in [0, 0.11]."""
    from paper_1412_8754_gb300 import surrogate as sg

    rng = np.random.default_rng(seed)
    G, H, D = 1024, 8, 16
    sset = dict(q=rng.uniform(0.0, 0.32, G), h=rng.uniform(0.025, 0.055, (G, H)),
                T=rng.uniform(0.0015, 0.0035, (G, H)), delta=rng.uniform(0.0, 0.11, (G, H, D)))
    sset["delta"][..., 0] = 0.0
    x, y = sg.training_data(ctx, N, sset)
    s, losses = sg.fit(ctx, x, y, epochs=120, batch=512, lr=2e-3, seed=seed)
    return s, float(np.sqrt(losses[-1]) * np.std(y)), losses


def test_ff_guided_scan_labels_are_exact(ff_oracle):
    """The FF scan guided by a surrogate trained on the FF model (grid: 8-point windows; golden:
    16-point windows; 5 q kept besides q = 0, margin 3 x the training RMS error).  On this small
    lattice the FF winners are lines whose own condensation is tiny (1e-9 .. 4e-6 per site, below
    the surrogate's resolution) but whose exact normal state lies 1.4e-5 .. 1.65e-5 per site below
    that of q = 0; the guided scan verifies such lines because of their exact normal state, so the
    labels and best q of every point, FF points included, are the oracle's.  (The normal states of
    most q lie below that of q = 0 by more than the margin here, so most lines are verified: the
    work saved is modest on this lattice, unlike on the large ones where the normal states agree.)"""
    c = workloads.ff_scan()
    N = c["N"]
    om, idx, star, labels, best = ff_oracle
    with ff_context(ffe.FFE_FP32C) as ctx:
        s, rms, losses = ff_surrogate(ctx, N, seed=3)
        res, glab, gbest, st = ffe.ffe_surrogate_scan(ctx.handle, s, N, c["qx"], c["qy"], c["h"], c["T"], n=c["n"],
                                                      lo=c["lo"], hi=c["hi"], window=8, q_keep=5, margin=3 * rms)
        gres, ggl, ggb, gst = ffe.ffe_surrogate_scan(ctx.handle, s, N, c["qx"], c["qy"], c["h"], c["T"], n=20,
                                                     lo=c["lo"], hi=c["hi"], window=16, q_keep=5, margin=3 * rms,
                                                     search=ffe.FFE_SEARCH_GOLDEN)
        full_g, flab_g, fbest_g = ctx.phase_scan(N, c["qx"], c["qy"], c["h"], c["T"], search=ffe.FFE_SEARCH_GOLDEN,
                                                 n=20, lo=c["lo"], hi=c["hi"])
        s.close()
    print(f"training RMS {rms:.3g} per site; grid: {st}; golden: {gst}")
    assert rms < 5e-6
    assert np.array_equal(glab, labels), (glab, labels)
    assert np.array_equal(gbest, best), (gbest, best)
    assert st["k_evals"] < st["k_evals_full"] and st["lines_pruned"] > 0, st
    kept = (res["flags"] & ffe.FFE_FLAG_PRUNED) == 0
    assert np.array_equal(res["idx_star"][kept & (res["idx_star"] > 0)], idx[kept & (res["idx_star"] > 0)])
    assert np.array_equal(ggl, flab_g) and np.array_equal(ggb, fbest_g), (ggl, flab_g, ggb, fbest_g)
    assert (ggl == search.FFLO).sum() >= 3
    assert gst["k_evals"] < gst["k_evals_full"] and gst["lines_pruned"] > 0, gst


def test_fflo_scan_u4_full_size_whole_lines():
    """The benchmark's FFLO scan plan at full size (N = 1024, 64 q x 32 h x 256 Delta, T = 0.002) at
    U = 4, where q = 0 and small q have interior BCS minima (Delta* ~ 0.115) up to h[11] = 0.053 and
    the first-order transition to the normal state lies before h[12] = 0.058.  On both sides the
    oracle evaluates the whole 256-point Delta grid of six q lines: each GPU argmin index is the
    oracle's; for every q of those two h the oracle's values at the GPU argmin and its neighbours
    give the GPU's label and best q."""
    cfg = workloads.fflo_scan()
    U, N, T = 4.0, cfg["N"], float(cfg["T"][0])
    grid = np.linspace(cfg["lo"], cfg["hi"], cfg["n"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as ctx:
        plan = ctx.plan_phase_scan(N, cfg["qx"], cfg["qy"], cfg["h"], cfg["T"], n=cfg["n"], lo=cfg["lo"],
                                   hi=cfg["hi"])
        plan.execute()
        res, labels, best = plan.fetch()
        plan.destroy()
    m = oracle.make_model(U=U)
    nq = len(cfg["qx"])
    seen_interior = 0
    for ih, want_label in ((11, search.BCS), (12, search.NORMAL)):
        for q in (0, 1, 2, 5, 20, 63):
            ref, _, _ = oracle.omega_batch(m, N, cfg["qx"][q], 0.0, cfg["h"][ih], T, grid)
            j = search.grid_argmin(ref)
            seen_interior += 0 < j < cfg["n"] - 1
            assert res["idx_star"][q, ih] == j, (ih, q, res["idx_star"][q, ih], j)
            assert per_site(res["omega_star"][q, ih], ref[j], N) <= TOL[ffe.FFE_FP32C]
            assert per_site(res["omega_lo"][q, ih], ref[0], N) <= TOL[ffe.FFE_FP32C]
        rows = []
        for q in range(nq):
            i = int(res["idx_star"][q, ih])
            rows += [(q, ii) for ii in sorted({0, max(i - 1, 0), i, min(i + 1, cfg["n"] - 1)})]
        Q = np.array([r[0] for r in rows])
        ref, _, _ = oracle.omega_batch(m, N, cfg["qx"][Q], 0.0, cfg["h"][ih], T, grid[[r[1] for r in rows]])
        val = {r: ref[k] for k, r in enumerate(rows)}
        star = np.array([val[(q, int(res["idx_star"][q, ih]))] for q in range(nq)])
        zero = np.array([val[(q, 0)] for q in range(nq)])
        for q in range(nq):
            i = int(res["idx_star"][q, ih])
            assert all(val[(q, i)] <= v for (qq, _), v in val.items() if qq == q), q
        want, wq = search.phase_label(star, zero, cfg["qx"] == 0.0)
        assert want == want_label
        assert labels[ih] == want and best[ih] == wq
    assert seen_interior >= 3


def test_fbz_scan_reaches_ff_on_a_2d_q_grid():
    """Alg. 1 over the whole Brillouin zone: the 64 x 64 Q grid of the FF model at N = 64 reduced to
    its 561-point wedge.  Every wedge line's argmin index is the oracle's, and the labels and best Q
    are those of the oracle over the wedge (an FF point among them, with Q on the grid's first
    shell); the full-grid labels follow from the symmetry pins of the oracle."""
    N, nq = 64, 64
    h = np.array([0.036, 0.04, 0.046])
    T = np.array([0.002])
    grid = np.linspace(0.0, 0.1, 41)
    w = qgrid.wedge(nq)
    q = 2.0 * math.pi * w / nq
    om, idx, star, labels, best = oracle_scan(ff_oracle_model(), N, q[:, 0], q[:, 1], h, T, grid)
    assert list(labels) == [search.BCS, search.FFLO, search.NORMAL], labels
    with ff_context(ffe.FFE_FP32C) as ctx:
        res, glab, gbq, wq = qgrid.fbz_phase_scan(ctx, N, nq, h, T, n=41, lo=0.0, hi=0.1)
    assert np.array_equal(wq, q)
    assert np.array_equal(res["idx_star"], idx)
    assert per_site(res["omega_star"], star, N).max() <= TOL[ffe.FFE_FP32C]
    assert np.array_equal(glab, labels)
    ok = best >= 0
    assert np.array_equal(gbq[ok], q[best[ok]])
    assert np.all(np.isnan(gbq[~ok]))
