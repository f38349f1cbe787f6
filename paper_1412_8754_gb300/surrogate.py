"""Training data and training runs of the learned surrogate (marshalling only).

The data are free energies computed by the library's own k-sum (ffe_omega) on
seeded parameter points; the target of a sample (q, h, T, Delta) is the
condensation energy per site (Omega(Delta) - Omega(0)) / N^2 of its line.
Training and inference run in the library's kernels (ffe_surrogate_*).
"""
from __future__ import annotations

import numpy as np

from . import ffe, workloads

N_PARAMS = ffe.N_SURROGATE_PARAMS
_FANS = [(4, 512), (None, 128), (128, 16384), (None, 128), (128, 16384), (None, 128), (128, 128), (None, 1)]


def initial_params(seed: int) -> np.ndarray:
    """Uniform(-sqrt(6/fan_in), +sqrt(6/fan_in)) weights, zero biases, seeded."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan, size in _FANS:
        if fan is None:
            parts.append(np.zeros(size))
        else:
            lim = np.sqrt(6.0 / fan)
            parts.append(rng.uniform(-lim, lim, size))
    return np.concatenate(parts).astype(np.float32)


def training_data(ctx: ffe.Context, N: int, sset: dict):
    """(x [n, 4] raw inputs, y [n] condensation energy per site) from ffe_omega."""
    q, h, T, d = sset["q"], sset["h"], sset["T"], sset["delta"]
    G, H, D = d.shape
    Q = np.broadcast_to(q[:, None, None], (G, H, D))
    HH = np.broadcast_to(h[:, :, None], (G, H, D))
    TT = np.broadcast_to(T[:, :, None], (G, H, D))
    om = ctx.omega(ffe.points(N, Q.ravel(), 0.0, HH.ravel(), TT.ravel(), d.ravel())).reshape(G, H, D)
    y = ffe.ffe_surrogate_targets(ctx.handle, om, N)
    x = np.stack([Q.ravel(), HH.ravel(), TT.ravel(), d.ravel()], axis=1)
    return x.astype(np.float32), y.ravel()


def fit(ctx: ffe.Context, x, y, epochs=30, batch=4096, lr=2e-3, seed=0, y_scale=None, decay=True):
    """A surrogate trained on (x, y) with Adam; returns (Surrogate, losses).  decay: the learning
    rate follows a half cosine from lr down to lr/50 over the epochs (one training call with a
    rate per epoch), so that the final weights settle instead of ending wherever constant-rate steps leave
    them."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(x))
    ys = float(y_scale) if y_scale else float(max(np.std(y), 1e-6))
    s = ffe.Surrogate(ctx, workloads.SURROGATE_SHIFT, workloads.SURROGATE_SCALE, ys, initial_params(seed))
    xp, yp = np.ascontiguousarray(x[perm]), np.ascontiguousarray(y[perm])
    if not decay:
        return s, s.train(xp, yp, epochs=epochs, batch=batch, lr=lr)
    e = np.arange(epochs)
    lrs = (lr * (0.02 + 0.98 * 0.5 * (1.0 + np.cos(np.pi * e / max(1, epochs - 1))))).astype(np.float32)
    return s, s.train_schedule(xp, yp, lrs, batch=batch)


def rms_error(s: "ffe.Surrogate", x, y, n=65536, seed=0) -> float:
    """RMS of prediction - target over a seeded subset of (x, y), in the target's units."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(x), size=min(n, len(x)), replace=False)
    return float(np.sqrt(np.mean((s.predict(x[pick]).astype(np.float64) - y[pick]) ** 2)))
