"""TEST INFRASTRUCTURE ONLY: plain FP64 reference of the learned closure's per-element
network (no counterpart in the paper; mandated on top of it): two GELU hidden layers,
y = W3 g(W2 g(W1 x + b1) + b2) + b3, g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, and the
mean-squared-error loss L = mean((y - t)^2) with its gradient by the chain rule.
The parameter layout is the flat vector W1, b1, W2, b2, W3, b3 (row-major, W_l [out][in])."""
import math

import numpy as np

_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unflatten(flat, n_in_pad, h1, h2, n_out):
    shapes = [("W1", (h1, n_in_pad)), ("b1", (h1,)), ("W2", (h2, h1)), ("b2", (h2,)), ("W3", (n_out, h2)),
              ("b3", (n_out,))]
    out, o = {}, 0
    for name, shape in shapes:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(p):
    return np.concatenate([p[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def forward(p, X):
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (z1, h1, z2, h2)


def loss_and_grad(p, X, T):
    """L = mean over rows and outputs of (y - t)^2 and dL/dp (same keys as p)."""
    y, (z1, h1, z2, h2) = forward(p, X)
    n = y.size
    L = float(((y - T) ** 2).sum() / n)
    dy = 2.0 * (y - T) / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dz2 = (dy @ p["W3"]) * gelu_grad(z2)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(axis=0)
    return L, g
