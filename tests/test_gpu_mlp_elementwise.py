"""The closure network's tensor-core kernels against the FP64 oracle network, element by element,
on the persistent multi-tile path that large problems take.

At the closure's size (884,736 elements) the persistent kernels (the resident-weight GEMM and the
fused three-layer forward) run dozens of 128-row tiles per CTA: both TMEM accumulators in turn and
the next tile's loads while the previous one drains. Here that path runs with a test-only grid cap
(2000 rows on 4 CTAs: 4 tiles each) and without one at 60,000 rows (469 tiles on one CTA per SM).

Bound, derived from the arithmetic (first-order error propagation through the network, evaluated
with the oracle's FP64 intermediate values; every stored activation and gradient is rounded to
BF16 once, unit roundoff U = 2^-9; every GEMM accumulates in FP32 with |error| <= F |A||B|,
F = 2e-5 for K <= 256, the bound the GEMM tests assert; GELU and its derivative are FP32
approximations with errors of 5e-7 |z| + 2^-23 |h| (tests/test_gelu_arith.py) and 1e-6):
  E_z1 = F (|W1||x| + |b1|),  E_h1 = U |h1| + |g'(z1)| E_z1 + eps_g,
  E_z2 = |W2| E_h1 + F (|W2||h1| + |b2|),  E_h2 = U |h2| + |g'(z2)| E_z2 + eps_g,
  E_y  = |W3| E_h2 + F (|W3||h2| + |b3|),
and through the backward pass the same way (dy, dz2, dz1 rounded to BF16; weight gradients
accumulated over the batch with F + B 2^-24). Every output and every gradient entry must lie
within 2 E of the oracle (the factor 2 covers the neglected second-order terms).
"""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1912_12059_gb300 import nsk

pytestmark = pytest.mark.gpu

U = 2.0 ** -9
F = 2e-5


def _bf16_round(a):
    import torch

    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _g2(z):
    """Second derivative of GELU, phi(z) (2 - z^2)."""
    return np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi) * (2.0 - z * z)


def _eps_g(z, h):
    return 5e-7 * np.abs(z) + 2.0 ** -23 * np.abs(h)


def forward_bound(p, X):
    """Oracle output y and the elementwise bound E_y; also the intermediates the backward bound uses."""
    y, (z1, h1, z2, h2) = omlp.forward(p, X)
    aX = np.abs(X)
    aW1, aW2, aW3 = (np.abs(p[k]) for k in ("W1", "W2", "W3"))
    E_z1 = F * (aX @ aW1.T + np.abs(p["b1"]))
    E_h1 = U * np.abs(h1) + np.abs(omlp.gelu_grad(z1)) * E_z1 + _eps_g(z1, h1)
    E_z2 = E_h1 @ aW2.T + F * (np.abs(h1) @ aW2.T + np.abs(p["b2"]))
    E_h2 = U * np.abs(h2) + np.abs(omlp.gelu_grad(z2)) * E_z2 + _eps_g(z2, h2)
    E_y = E_h2 @ aW3.T + F * (np.abs(h2) @ aW3.T + np.abs(p["b3"]))
    return y, E_y, dict(z1=z1, h1=h1, z2=z2, h2=h2, E_z1=E_z1, E_h1=E_h1, E_z2=E_z2, E_h2=E_h2)


def gradient_bound(p, X, T):
    """Oracle loss gradient (keys W1..b3) and its elementwise bounds."""
    y, E_y, it = forward_bound(p, X)
    _, g = omlp.loss_and_grad(p, X, T)
    B, n = y.shape[0], y.size
    FB = F + B * 2.0 ** -24
    aW2, aW3 = np.abs(p["W2"]), np.abs(p["W3"])
    z1, h1, z2, h2 = it["z1"], it["h1"], it["z2"], it["h2"]
    dy = 2.0 * (y - T) / n
    E_gf = 2.0 / n * E_y                      # the FP32 output gradient (before its BF16 copy)
    E_dy = U * np.abs(dy) + E_gf
    a2 = dy @ p["W3"]
    E_a2 = E_dy @ aW3 + F * (np.abs(dy) @ aW3)
    dz2 = a2 * omlp.gelu_grad(z2)
    E_dz2f = np.abs(omlp.gelu_grad(z2)) * E_a2 + np.abs(a2) * (np.abs(_g2(z2)) * it["E_z2"] + 1e-6)
    E_dz2 = U * np.abs(dz2) + E_dz2f
    a1 = dz2 @ p["W2"]
    E_a1 = E_dz2 @ aW2 + F * (np.abs(dz2) @ aW2)
    dz1 = a1 * omlp.gelu_grad(z1)
    E_dz1f = np.abs(omlp.gelu_grad(z1)) * E_a1 + np.abs(a1) * (np.abs(_g2(z1)) * it["E_z1"] + 1e-6)
    E_dz1 = U * np.abs(dz1) + E_dz1f
    aX = np.abs(X)
    E = {"W3": E_dy.T @ np.abs(h2) + np.abs(dy).T @ it["E_h2"] + FB * (np.abs(dy).T @ np.abs(h2)),
         "b3": E_gf.sum(axis=0) + FB * np.abs(dy).sum(axis=0),
         "W2": E_dz2.T @ np.abs(h1) + np.abs(dz2).T @ it["E_h1"] + FB * (np.abs(dz2).T @ np.abs(h1)),
         "b2": E_dz2f.sum(axis=0) + FB * np.abs(dz2).sum(axis=0),
         "W1": E_dz1.T @ aX + FB * (np.abs(dz1).T @ aX),
         "b1": E_dz1f.sum(axis=0) + FB * np.abs(dz1).sum(axis=0)}
    return g, E


def _network(n_in, h1, h2, n_out, max_batch, max_rows, seed):
    m = nsk.MLP(n_in, h1, h2, n_out, max_batch=max_batch, max_rows=max_rows)
    m.init_params(seed=seed)
    p = omlp.unflatten(m.get_params().astype(np.float64), m.n_in_pad, h1, h2, n_out)
    for k in ("W1", "W2", "W3"):
        p[k] = _bf16_round(p[k])  # the GPU multiplies BF16 copies of the weights
    return m, p


def _inputs(rows, n_in, n_in_pad, seed, gpu):
    import torch

    rng = np.random.default_rng(seed)
    Xn = np.zeros((rows, n_in_pad))
    Xn[:, :n_in] = rng.uniform(-1, 1, size=(rows, n_in))
    Xt = torch.from_numpy(Xn).to(torch.bfloat16)
    return Xt.to(gpu), Xt.double().numpy(), rng


@pytest.fixture
def grid_cap():
    """Set a test-only cap on the persistent tensor-core grids; always removed afterwards."""
    caps = []

    def set_cap(c):
        nsk._test_hook_tc_grid_cap(c)
        caps.append(c)

    yield set_cap
    nsk._test_hook_tc_grid_cap(0)


@pytest.mark.parametrize("rows,cap", [(2000, 4), (2000, 3), (60000, 0)])
@pytest.mark.parametrize("fused", [True, False])
def test_forward_elementwise_on_multi_tile_path(gpu, grid_cap, rows, cap, fused):
    """Inference forward of the closure's network (140 -> 256 -> 256 -> 64), fused kernel and the
    three GEMMs, with several row tiles per CTA (and a ragged last tile: 2000 = 15 x 128 + 80)."""
    import torch

    m, p = _network(140, 256, 256, 64, 256, rows, seed=11)
    m.set_fused_forward(fused)
    X, Xq, _ = _inputs(rows, 140, m.n_in_pad, 12, gpu)
    grid_cap(cap)
    Y = torch.full((rows, 64), float("nan"), dtype=torch.float32, device=gpu)
    m.forward(X, Y)
    torch.cuda.synchronize()
    got = Y.cpu().double().numpy()
    y_ref, E_y, _ = forward_bound(p, Xq)
    assert np.isfinite(got).all()
    viol = np.abs(got - y_ref) > 2.0 * E_y
    assert not viol.any(), (int(viol.sum()), float((np.abs(got - y_ref) / E_y).max()))
    m.close()


@pytest.mark.parametrize("B,cap", [(2000, 4), (512, 0)])
def test_gradients_elementwise_on_multi_tile_path(gpu, grid_cap, B, cap):
    """Loss and every gradient block of the training pass (forward GEMMs with the GELU epilogue,
    backward GEMMs with the GELU-derivative epilogue, split-K weight gradients), the training
    GEMMs running several row tiles per CTA (B = 2000 on 4 CTAs)."""
    import torch

    m, p = _network(140, 256, 256, 64, B, B, seed=13)
    X, Xq, rng = _inputs(B, 140, m.n_in_pad, 14, gpu)
    Tn = rng.normal(size=(B, 64)) * 0.5
    T = torch.from_numpy(Tn).float().to(gpu)
    grid_cap(cap)
    g_gpu, loss = m.gradients(X, T)
    L_ref, _ = omlp.loss_and_grad(p, Xq, Tn)
    assert abs(loss - L_ref) <= 1e-2 * L_ref
    g_ref, E = gradient_bound(p, Xq, Tn)
    gg = m.unflatten(g_gpu.astype(np.float64))
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, b, e = gg[k], g_ref[k], E[k]
        if k == "W1":
            assert np.abs(a[:, 140:]).max() == 0.0  # padded inputs carry no gradient
            a, b, e = a[:, :140], b[:, :140], e[:, :140]
        viol = np.abs(a - b) > 2.0 * e
        assert not viol.any(), (k, int(viol.sum()), float((np.abs(a - b) / e).max()))
    m.close()


def test_grid_cap_leaves_results_unchanged(gpu, grid_cap):
    """The cap changes the schedule only: the same outputs bit for bit."""
    import torch

    m, _ = _network(140, 256, 256, 64, 256, 2000, seed=15)
    X, _, _ = _inputs(2000, 140, m.n_in_pad, 16, gpu)
    Y0 = torch.empty((2000, 64), dtype=torch.float32, device=gpu)
    Y1 = torch.empty_like(Y0)
    m.forward(X, Y0)
    grid_cap(2)
    m.forward(X, Y1)
    torch.cuda.synchronize()
    assert torch.equal(Y0, Y1)
    m.close()


@pytest.fixture
def fwd_kernel():
    """Select the fused forward's kernel through the test hook; always reset to the default."""
    yield lambda which: nsk._test_hook_mlp_fwd_kernel(which)
    nsk._test_hook_mlp_fwd_kernel(0)


@pytest.mark.parametrize("n_in,h1,h2,n_out,rows,cap", [(140, 256, 256, 64, 2000, 3), (140, 256, 256, 64, 60000, 0),
                                                      (40, 64, 128, 32, 300, 1), (70, 128, 256, 16, 1000, 2),
                                                      (24, 48, 80, 16, 777, 2)])
def test_warp_specialised_forward_equals_serial_kernel(gpu, grid_cap, fwd_kernel, n_in, h1, h2, n_out, rows, cap):
    """The warp-specialised forward (operands by TMA, load, MMA and epilogue stages overlapped across
    activation chunks and row tiles) issues the same MMAs in the same K order with the same epilogue
    arithmetic as the stage-by-stage kernel: the same outputs bit for bit, with several row tiles
    per CTA, a ragged last tile, and hidden widths that are not multiples of its 64-column chunk."""
    import torch

    m, p = _network(n_in, h1, h2, n_out, 256, rows, seed=21)
    m.set_fused_forward(True)
    X, Xq, _ = _inputs(rows, n_in, m.n_in_pad, 22, gpu)
    grid_cap(cap)
    Ys = torch.full((rows, n_out), float("nan"), dtype=torch.float32, device=gpu)
    Yw = torch.full((rows, n_out), float("nan"), dtype=torch.float32, device=gpu)
    fwd_kernel(1)
    m.forward(X, Ys)
    fwd_kernel(0)
    m.forward(X, Yw)
    torch.cuda.synchronize()
    assert torch.isfinite(Yw).all()
    assert torch.equal(Ys, Yw), float((Ys - Yw).abs().max())
    if rows <= 2000:  # and both within the elementwise bound of the oracle network
        y_ref, E_y, _ = forward_bound(p, Xq)
        got = Yw.cpu().double().numpy()
        assert not (np.abs(got - y_ref) > 2.0 * E_y).any()
    m.close()
