"""Pins of the FP64 surrogate MLP reference: backprop vs central finite differences."""
import numpy as np

from oracle import mlp

RNG = np.random.default_rng(3)


def test_parameter_count():
    assert mlp.N_PARAMS == 33793
    theta = mlp.init_params(1)
    assert theta.size == mlp.N_PARAMS
    assert np.allclose(mlp.pack(mlp.unpack(theta)), theta)


def test_silu_derivative_by_differences():
    z = RNG.normal(0, 3, 1000)
    eps = 1e-6
    num = (mlp.silu(z + eps) - mlp.silu(z - eps)) / (2 * eps)
    assert np.max(np.abs(num - mlp.silu_prime(z))) < 1e-8


def test_backprop_matches_finite_differences():
    theta = mlp.init_params(5) * 0.5
    x = RNG.uniform(0, 1, (16, 4))
    t = RNG.normal(0, 1, 16)
    _, g = mlp.loss_and_grad(theta, x, t)
    idx = np.concatenate([RNG.choice(np.arange(s, e), 12, replace=False) for s, e in
                          [(0, 512), (512, 640), (640, 17024), (17024, 17152), (17152, 33536),
                           (33536, 33664), (33664, 33792)]] + [np.array([33792])])
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp, _ = mlp.loss_and_grad(tp, x, t)
        lm, _ = mlp.loss_and_grad(tm, x, t)
        num = (lp - lm) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_adam_reduces_a_quadratic():
    target = RNG.normal(0, 1, 50)
    theta = np.zeros(50)
    opt = mlp.Adam(50, lr=0.05)
    for _ in range(500):
        theta = opt.step(theta, 2 * (theta - target))
    assert np.max(np.abs(theta - target)) < 1e-2


def test_adam_first_step_is_lr_times_sign():
    """Bias correction makes the first update lr * g / (|g| + eps)."""
    g = RNG.normal(0, 1, 20)
    opt = mlp.Adam(20, lr=1e-3)
    theta = opt.step(np.zeros(20), g)
    assert np.allclose(theta, -1e-3 * np.sign(g), atol=1e-9)
