"""Pins of the closure's reference pieces (no GPU).

1. The FP64 network reference (oracle/mlp.py): gradients equal central finite
   differences of its own loss; forward pass, loss and gradients equal PyTorch's float64
   layers, mse_loss and autograd.
2. The closure target: the steady state of the oracle's c equation at frozen rho
   (v = 0) is the quasi-equilibrium of the Korteweg-limit remark (Sec. 2.3),
   c - (kappa/alpha) c_xx = rho. For rho = rho0 + A sin(2 pi x) on the periodic unit
   interval the exact solution is c = rho0 + A sin(2 pi x) / (1 + (kappa/alpha)(2 pi)^2);
   the discrete steady state converges to it under mesh refinement.
"""
import math

import numpy as np

import oracle as O
from oracle import mlp


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    shapes = dict(n_in_pad=16, h1=16, h2=16, n_out=8)
    flat = rng.normal(size=16 * 16 + 16 + 16 * 16 + 16 + 8 * 16 + 8) * 0.3
    X = rng.normal(size=(7, 16))
    T = rng.normal(size=(7, 8))
    p = mlp.unflatten(flat, **shapes)
    _, g = mlp.loss_and_grad(p, X, T)
    gf = mlp.flatten(g)
    for i in rng.choice(flat.size, 40, replace=False):
        e = np.zeros_like(flat)
        e[i] = 1e-6
        lp = mlp.loss_and_grad(mlp.unflatten(flat + e, **shapes), X, T)[0]
        lm = mlp.loss_and_grad(mlp.unflatten(flat - e, **shapes), X, T)[0]
        assert abs((lp - lm) / 2e-6 - gf[i]) < 1e-7 * max(1.0, abs(gf[i]))


def test_mlp_matches_torch_autograd():
    """The forward pass, the mean-squared-error loss and its gradient equal PyTorch's float64
    Linear layers with the exact (erf) GELU, mse_loss (mean over every output) and autograd."""
    torch = __import__("torch")
    rng = np.random.default_rng(3)
    shapes = dict(n_in_pad=16, h1=24, h2=20, n_out=8)
    n = 24 * 16 + 24 + 20 * 24 + 20 + 8 * 20 + 8
    flat = rng.normal(size=n) * 0.3
    X = rng.normal(size=(9, 16))
    T = rng.normal(size=(9, 8))
    p = mlp.unflatten(flat, **shapes)
    y, _ = mlp.forward(p, X)
    L, g = mlp.loss_and_grad(p, X, T)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    tX, tT = torch.tensor(X, dtype=torch.float64), torch.tensor(T, dtype=torch.float64)
    F = torch.nn.functional
    h = F.gelu(F.linear(tX, tp["W1"], tp["b1"]), approximate="none")
    h = F.gelu(F.linear(h, tp["W2"], tp["b2"]), approximate="none")
    ty = F.linear(h, tp["W3"], tp["b3"])
    tL = F.mse_loss(ty, tT)
    tL.backward()
    assert np.allclose(y, ty.detach().numpy(), rtol=1e-13, atol=1e-14)
    assert abs(L - tL.item()) < 1e-14 * max(1.0, abs(L))
    for k in p:
        assert np.allclose(g[k], tp[k].grad.numpy(), rtol=1e-12, atol=1e-15), k


def test_gelu_closed_forms():
    assert abs(mlp.gelu(np.array([0.0]))[0]) == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15  # Phi(1)
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


def _steady_c(E, N, kappa, alpha, rho0=1.2, A=0.1):
    orc = O.Oracle(1, (E,), (0.0,), (1.0,), N, O.NODES_GAUSS, kappa=kappa, alpha=alpha, beta=1.0, mu=0.0)
    x = orc.coords()[0]
    U = np.zeros(orc.shape)
    U[0] = rho0 + A * np.sin(2 * math.pi * x)

    def Rc(c):
        V = U.copy()
        V[2] = c.reshape(U[2].shape)
        return orc.rhs(V)[2].ravel()

    n = U[2].size
    r0 = Rc(np.zeros(n))
    M = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = Rc(e) - r0
    c = np.linalg.solve(M, -r0)
    exact = rho0 + A * np.sin(2 * math.pi * x.ravel()) / (1.0 + kappa / alpha * (2 * math.pi) ** 2)
    return float(np.abs(c - exact).max())


def test_c_equation_steady_state_is_screened_poisson():
    # BR1 with odd N converges at order about N in the maximum norm (observed 2.6 .. 3.0 for N = 3)
    errs = [_steady_c(E, 3, kappa=1e-3, alpha=1.0) for E in (4, 8, 16, 32)]
    assert errs[-1] < 3e-7
    assert all(errs[i] / errs[i + 1] > 5.5 for i in range(3)), errs
