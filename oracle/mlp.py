"""FP64 reference of the surrogate MLP (test infrastructure only).

Network 4 -> 128 -> 128 -> 128 -> 1 with SiLU activations, inputs
(q, h, T, Delta) mapped affinely to [0, 1], output the condensation energy per
site (Omega(Delta) - Omega(0)) / N^2 divided by a fixed target scale.  The
paper has no learned component; this module is the independent reference for
the hand-written training kernels: forward pass, backward pass written out by
hand (chain rule, no autodiff), mean-squared-error loss and the Adam update
(Kingma & Ba 2015, bias-corrected).  Pinned by central finite differences in
tests/test_oracle_mlp.py.

Flat parameter layout (33 793 floats):
  W1 [4][128], b1 [128], W2 [128][128], b2 [128], W3 [128][128], b3 [128],
  W4 [128], b4 [1]; W[i][o] maps input i to output o.
"""
from __future__ import annotations

import numpy as np

WIDTH = 128
SIZES = [("W1", (4, WIDTH)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
         ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("W4", (WIDTH,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)

# Input box of the surrogate: q in [0, 0.2 pi], h in [0, 0.15], T in [0.001, 0.03], Delta in [0, 0.2]
SHIFT = np.array([0.0, 0.0, 0.001, 0.0])
SCALE = 1.0 / np.array([0.2 * np.pi, 0.15, 0.029, 0.2])


def unpack(theta):
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed=0):
    """He-style uniform initialisation, seeded."""
    rng = np.random.default_rng(seed)
    parts = {}
    fan = {"W1": 4, "W2": WIDTH, "W3": WIDTH, "W4": WIDTH}
    for name, shape in SIZES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / fan[name])
            parts[name] = rng.uniform(-lim, lim, size=shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def silu_prime(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def features(raw):
    """raw [n, 4] = (q, h, T, Delta) -> normalised inputs."""
    return (np.asarray(raw, dtype=np.float64) - SHIFT) * SCALE


def forward(theta, x):
    """x: normalised inputs [n, 4].  Returns (y [n], cache)."""
    p = unpack(theta)
    z1 = x @ p["W1"] + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = silu(z2)
    z3 = h2 @ p["W3"] + p["b3"]
    h3 = silu(z3)
    y = h3 @ p["W4"] + p["b4"][0]
    return y, (x, z1, h1, z2, h2, z3, h3)


def loss_and_grad(theta, x, t):
    """Mean squared error over the batch and its gradient (hand-written backprop)."""
    p = unpack(theta)
    y, (x, z1, h1, z2, h2, z3, h3) = forward(theta, x)
    n = x.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n                                # dL/dy
    g = {"W4": h3.T @ dy, "b4": np.array([dy.sum()])}
    dz3 = np.outer(dy, p["W4"]) * silu_prime(z3)    # dL/dz3
    g["W3"] = h2.T @ dz3
    g["b3"] = dz3.sum(axis=0)
    dz2 = (dz3 @ p["W3"].T) * silu_prime(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * silu_prime(z1)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


class Adam:
    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
