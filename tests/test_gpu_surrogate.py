"""The surrogate's hand-written training and inference kernels vs the FP64 MLP reference.

Tolerances reflect the kernels' BF16 tensor-core products with FP32 accumulation:
predictions and gradients agree with the FP64 reference to ~1 % (norm-wise)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1412_8754_gb300 import ffe

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(2024)
Y_SCALE = 0.01


def raw_inputs(n, rng=RNG):
    lo = np.array([0.0, 0.0, 0.001, 0.0])
    hi = np.array([0.2 * np.pi, 0.15, 0.03, 0.2])
    return lo + (hi - lo) * rng.uniform(0, 1, (n, 4))


@pytest.fixture(scope="module")
def ctx():
    c = ffe.Context(prec=ffe.FFE_FP32C)
    yield c
    c.close()


def make(ctx, theta):
    return ffe.Surrogate(ctx, mlp.SHIFT, mlp.SCALE, Y_SCALE, theta.astype(np.float32))


def test_forward_matches_reference(ctx):
    theta = mlp.init_params(11)
    s = make(ctx, theta)
    xr = raw_inputs(1000)
    got = s.predict(xr)
    ref, _ = mlp.forward(theta.astype(np.float32).astype(np.float64), mlp.features(xr))
    ref = ref * Y_SCALE
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 3e-2, err  # BF16 activations and weights: 2^-9 relative rounding per value
    s.close()


@pytest.mark.parametrize("n", [200, 64, 1024])
def test_gradient_matches_reference(ctx, n):
    theta = mlp.init_params(12)
    s = make(ctx, theta)
    xr = raw_inputs(n)
    t = RNG.normal(0, 1, n) * Y_SCALE
    loss, g = s.grad(xr, t)
    lref, gref = mlp.loss_and_grad(theta.astype(np.float32).astype(np.float64), mlp.features(xr), t / Y_SCALE)
    assert abs(loss - lref) <= 1e-2 * lref
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert rel < 2e-2 and cos > 0.999, (rel, cos)
    # every parameter block gets its gradient (W1, b1, W2, b2, W3, b3, W4, b4)
    for a, b in [(0, 512), (512, 640), (640, 17024), (17024, 17152), (17152, 33536), (33536, 33664),
                 (33664, 33792), (33792, 33793)]:
        rb = np.linalg.norm(g[a:b] - gref[a:b]) / max(np.linalg.norm(gref[a:b]), 1e-30)
        assert rb < 5e-2, (a, b, rb)
    s.close()


def test_first_adam_step_matches_reference(ctx):
    theta = mlp.init_params(13)
    s = make(ctx, theta)
    xr = raw_inputs(256)
    t = RNG.normal(0, 1, 256) * Y_SCALE
    s.train(xr, t, epochs=1, batch=256, lr=1e-3)
    new = s.get_params().astype(np.float64)
    _, gref = mlp.loss_and_grad(theta.astype(np.float32).astype(np.float64), mlp.features(xr), t / Y_SCALE)
    opt = mlp.Adam(mlp.N_PARAMS, lr=1e-3)
    want = opt.step(theta.astype(np.float32).astype(np.float64), gref)
    big = np.abs(gref) > 1e-3 * np.abs(gref).max()
    # the first bias-corrected step is lr * sign(g) wherever g is not tiny
    assert np.mean(np.abs(new[big] - want[big]) < 1e-6) > 0.99
    s.close()


def test_training_fits_a_smooth_target(ctx):
    """Adam on the GPU kernels drives the loss of a smooth synthetic target down."""
    rng = np.random.default_rng(5)
    xr = raw_inputs(16384, rng)
    f = mlp.features(xr)
    t = (np.sin(3 * f[:, 0]) * f[:, 3] ** 2 - 0.5 * f[:, 1] * f[:, 3] + 0.2 * f[:, 2]) * Y_SCALE
    s = make(ctx, mlp.init_params(14))
    losses = s.train(xr, t, epochs=30, batch=512, lr=2e-3)
    assert losses[-1] < 0.05 * losses[0], losses
    pred = s.predict(xr[:2000])
    rms = np.sqrt(np.mean((pred - t[:2000]) ** 2)) / np.std(t)
    assert rms < 0.1, rms
    s.close()


def test_guided_scan_with_full_window_is_the_full_scan(ctx):
    """window = whole grid, every q kept: the guided scan reduces to the grid scan."""
    from paper_1412_8754_gb300 import surrogate as sg

    N, U = 32, 4.0
    qx = np.array([0.0, 0.15, 0.3, 0.45])
    h = np.array([0.0, 0.07, 0.14])
    T = np.array([0.004, 0.02])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as c:
        s = ffe.Surrogate(c, mlp.SHIFT, mlp.SCALE, Y_SCALE, sg.initial_params(3))
        res, lab, best, st = ffe.ffe_surrogate_scan(c.handle, s, N, qx, np.zeros(4), h, T, n=33,
                                                    window=33, q_keep=3)
        ref, rlab, rbest = c.phase_scan(N, qx, np.zeros(4), h, T, n=33)
        s.close()
    assert np.array_equal(res["idx_star"], ref["idx_star"])
    assert np.array_equal(lab, rlab) and np.array_equal(best, rbest)
    assert st["fallbacks"] == 0 and st["lines_pruned"] == 0
    assert st["k_evals"] == st["k_evals_full"]  # no margin: no normal-state pass


def test_guided_golden_with_whole_range_window_is_the_golden_scan(ctx):
    """window = the whole prediction grid, every q kept: each line's bracket is [lo, hi] with the
    full number of reductions, so the guided golden scan is the golden scan."""
    from paper_1412_8754_gb300 import surrogate as sg

    N, U, steps = 32, 4.0, 12
    qx = np.array([0.0, 0.2, 0.4])
    h = np.array([0.0, 0.05, 0.1])
    T = np.array([0.004, 0.015])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as c:
        s = ffe.Surrogate(c, mlp.SHIFT, mlp.SCALE, Y_SCALE, sg.initial_params(4))
        res, lab, best, st = ffe.ffe_surrogate_scan(c.handle, s, N, qx, np.zeros(3), h, T, n=steps, window=256,
                                                    q_keep=2, search=ffe.FFE_SEARCH_GOLDEN)
        ref, rlab, rbest = c.phase_scan(N, qx, np.zeros(3), h, T, search=ffe.FFE_SEARCH_GOLDEN, n=steps)
        s.close()
    assert np.array_equal(lab, rlab) and np.array_equal(best, rbest)
    np.testing.assert_array_equal(res["delta_star"], ref["delta_star"])
    np.testing.assert_allclose(res["omega_star"], ref["omega_star"], rtol=0, atol=1e-9 * N * N)
    assert st["fallbacks"] == 0 and st["lines_pruned"] == 0
    assert st["k_evals"] == st["k_evals_full"]


def test_guided_golden_rescans_every_line_of_a_flagged_point(ctx):
    """An untrained surrogate places the windows arbitrarily and a huge margin flags every line
    predicted at Delta = lo; no q is pruned.  A flagged point is scanned again with all its
    verified lines over the whole range (a line left on its window there would get no edge
    check), the others fall back on their window edges: labels and best q are the golden
    scan's."""
    from paper_1412_8754_gb300 import surrogate as sg

    N, U, steps = 32, 4.0, 12
    qx = np.array([0.0, 0.2, 0.4])
    h = np.array([0.0, 0.05, 0.1, 0.15])
    T = np.array([0.004, 0.015])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as c:
        ref, rlab, rbest = c.phase_scan(N, qx, np.zeros(3), h, T, search=ffe.FFE_SEARCH_GOLDEN, n=steps)
        for seed in (5, 6, 7):
            s = ffe.Surrogate(c, mlp.SHIFT, mlp.SCALE, Y_SCALE, sg.initial_params(seed))
            res, lab, best, st = ffe.ffe_surrogate_scan(c.handle, s, N, qx, np.zeros(3), h, T, n=steps, window=16,
                                                        q_keep=2, margin=1e3, search=ffe.FFE_SEARCH_GOLDEN)
            s.close()
            assert st["lines_pruned"] == 0
            assert np.array_equal(lab, rlab) and np.array_equal(best, rbest), (seed, lab, rlab, best, rbest)


def test_trained_surrogate_guides_the_scan():
    """A surrogate trained on the library's own free energies cuts the exact work of a
    grid scan while finding the full scan's minima and labels; an untrained one does not."""
    from paper_1412_8754_gb300 import surrogate as sg
    from paper_1412_8754_gb300 import workloads

    N, U, n = 32, 4.0, 41
    qx = np.linspace(0.0, 0.2 * np.pi, 6)
    h = np.linspace(0.0, 0.15, 6)
    T = np.array([0.003, 0.01, 0.02])
    with ffe.Context(prec=ffe.FFE_FP32C, U=U) as c:
        sset = workloads.surrogate_set(n_groups=512, n_ht=8, n_delta=16, seed=7, T_hi=0.02)
        x, y = sg.training_data(c, N, sset)
        trained, losses = sg.fit(c, x, y, epochs=60, batch=512, lr=2e-3, seed=1)
        untrained = ffe.Surrogate(c, workloads.SURROGATE_SHIFT, workloads.SURROGATE_SCALE, trained_scale(y),
                                  sg.initial_params(1))
        ref, rlab, rbest = c.phase_scan(N, qx, np.zeros_like(qx), h, T, n=n)
        out = {}
        for name, s in (("trained", trained), ("untrained", untrained)):
            res, lab, best, st = ffe.ffe_surrogate_scan(c.handle, s, N, qx, np.zeros_like(qx), h, T, n=n,
                                                        window=8, q_keep=2)
            out[name] = (res, lab, st)
        # with a margin of three training RMS errors every q the surrogate cannot order against
        # the best is kept: the labels and best q are the full scan's
        rms = float(np.sqrt(losses[-1]) * trained_scale(y))
        mres, mlab, mbest, mst = ffe.ffe_surrogate_scan(c.handle, trained, N, qx, np.zeros_like(qx), h, T, n=n,
                                                        window=8, q_keep=2, margin=3 * rms)
        # golden-section form: windows bracketed, fewer reductions, labels of the full golden scan
        gref, glab_ref, gbest_ref = c.phase_scan(N, qx, np.zeros_like(qx), h, T, search=ffe.FFE_SEARCH_GOLDEN,
                                                 n=20)
        gres, glab, _, gst = ffe.ffe_surrogate_scan(c.handle, trained, N, qx, np.zeros_like(qx), h, T, n=20,
                                                    window=16, q_keep=2, search=ffe.FFE_SEARCH_GOLDEN)
        _, mglab, mgbest, _ = ffe.ffe_surrogate_scan(c.handle, trained, N, qx, np.zeros_like(qx), h, T, n=20,
                                                     window=16, q_keep=2, margin=3 * rms,
                                                     search=ffe.FFE_SEARCH_GOLDEN)
        trained.close()
        untrained.close()
    assert losses[-1] < 0.1 * losses[0]
    # without a margin two q whose predicted minima lie within the surrogate's error of each
    # other may be ordered wrongly and the better one pruned, so a few labels may differ ...
    res, lab, st = out["trained"]
    agree_labels = np.mean(lab == rlab)
    # ... with the margin none does
    assert np.array_equal(mlab, rlab) and np.array_equal(mbest, rbest), (mlab, rlab)
    assert mst["k_evals"] < st["k_evals_full"], mst
    kept = np.zeros_like(ref["idx_star"], dtype=bool)
    found = res["idx_star"] == ref["idx_star"]
    assert agree_labels >= 0.9, (lab, rlab)
    assert st["k_evals"] < 0.5 * st["k_evals_full"], st
    pruned = (res["flags"] & ffe.FFE_FLAG_PRUNED) != 0
    assert pruned.sum() == st["lines_pruned"] > 0
    assert np.all(res["idx_star"][pruned] == 0)
    # the trained network predicts the exact condensation energies better than chance
    assert st["rms_error"] < out["untrained"][2]["rms_error"], (st, out["untrained"][2])
    assert np.mean(found | (ref["idx_star"] == 0)) >= 0.5
    assert np.mean(glab == glab_ref) >= 0.9, (glab, glab_ref)
    assert np.array_equal(mglab, glab_ref) and np.array_equal(mgbest, gbest_ref), (mglab, glab_ref)
    assert gst["k_evals"] < 0.75 * gst["k_evals_full"], gst  # q = 0 and 2 of 5 other q are kept
    gpruned = (gres["flags"] & ffe.FFE_FLAG_PRUNED) != 0
    assert gpruned.sum() == gst["lines_pruned"] > 0
    # a kept line whose minimum lies inside its window finds the full search's minimum
    both = ~gpruned & ((gref["flags"] & ffe.FFE_FLAG_LOWER) == 0) & ((gres["flags"] & ffe.FFE_FLAG_LOWER) == 0)
    assert both.sum() > 0
    np.testing.assert_allclose(gres["delta_star"][both], gref["delta_star"][both], atol=2e-3)


def trained_scale(y):
    return float(max(np.std(y), 1e-6))


def test_checkpoint_resumes_training_bit_for_bit(ctx):
    """Save after two epochs, train two more; load the checkpoint into a fresh surrogate (other
    weights, other maps) and train the same two epochs: the same losses and weights, bit for bit."""
    rng = np.random.default_rng(9)
    xr = raw_inputs(4096, rng)
    f = mlp.features(xr)
    t = (np.sin(3 * f[:, 0]) * f[:, 3] ** 2 - 0.5 * f[:, 1] * f[:, 3]) * Y_SCALE
    s = make(ctx, mlp.init_params(21))
    s.train(xr, t, epochs=2, batch=512, lr=2e-3)
    ckpt = s.save()
    la = s.train(xr, t, epochs=2, batch=512, lr=2e-3)
    wa = s.get_params()
    s.close()
    r = ffe.Surrogate(ctx, np.zeros(4), np.ones(4), 1.0, mlp.init_params(22).astype(np.float32))
    r.load(ckpt)
    lb = r.train(xr, t, epochs=2, batch=512, lr=2e-3)
    wb = r.get_params()
    with pytest.raises(ffe.FFEError):
        r.load(ckpt[:100])
    r.close()
    assert np.array_equal(la, lb) and np.array_equal(wa, wb)


@pytest.mark.parametrize("N", [512, 24])
def test_training_targets_are_the_condensation_energies(ctx, N):
    """ffe_surrogate_targets: (omega[l, j] - omega[l, 0]) / N^2 per line, rounded once to FP32 from
    the FP64 difference and quotient (IEEE: the same bits as numpy's), on a ragged line count."""
    rng = np.random.default_rng(N)
    om = -1.7 * N * N + rng.normal(0.0, 1e-3 * N * N, (37, 5, 16))
    got = ffe.ffe_surrogate_targets(ctx.handle, om, N)
    want = ((om - om[..., :1]) / float(N) ** 2).astype(np.float32)
    assert got.dtype == np.float32 and got.shape == om.shape
    assert np.array_equal(got, want)
    assert np.all(got[..., 0] == 0.0)


def test_learning_rate_schedule_equals_one_call_per_epoch(ctx):
    """ffe_surrogate_train_schedule with rates r[0..2] gives the same losses and weights, bit for
    bit, as three one-epoch ffe_surrogate_train calls at r[e] (the Adam step count carries over)."""
    rng = np.random.default_rng(31)
    xr = raw_inputs(3000, rng)
    f = mlp.features(xr)
    t = (np.cos(2 * f[:, 0]) * f[:, 3] ** 2 + 0.3 * f[:, 2] * f[:, 3]) * Y_SCALE
    lrs = np.array([3e-3, 1.5e-3, 2e-4], dtype=np.float32)
    a = make(ctx, mlp.init_params(41))
    la = np.array([a.train(xr, t, epochs=1, batch=256, lr=float(r))[0] for r in lrs], dtype=np.float32)
    wa = a.get_params()
    a.close()
    b = make(ctx, mlp.init_params(41))
    lb = b.train_schedule(xr, t, lrs, batch=256)
    wb = b.get_params()
    with pytest.raises(ffe.FFEError):
        b.train_schedule(xr, t, np.array([1e-3, 0.0], dtype=np.float32), batch=256)
    b.close()
    assert np.array_equal(la, lb) and np.array_equal(wa, wb)
    assert lb[-1] < lb[0]
