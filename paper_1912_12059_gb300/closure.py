"""Learned c-closure: training data from the method's own explicit runs, and training.

The quasi-equilibrium of the relaxation variable (the Korteweg-limit remark of
Sec. 2.3: c - (kappa/alpha) Lap c = rho, reached after t >> beta/alpha) is what
the explicit c equation tracks; the per-element network learns it from (rho, c)
snapshots of explicit runs and replaces the stiff c equation (include/nsk.h:
nsk_set_closure). Targets are scaled to the reference element,
y = (c - rho) / ((kappa/alpha)(2/h)^2), which is O(1) and independent of the
mesh size at leading order (it approximates the reference-element Laplacian of
rho). Every computation runs in libnsk.so; this module only orchestrates calls.
"""
from __future__ import annotations

import math

import numpy as np


def collect_snapshots(solver, dt, first_step, every, count, interface_frac=0.85, rng=None, max_per_snapshot=None):
    """Advance `solver` (explicit c equation) and gather (features, targets) of elements.

    Elements are drawn per snapshot with probability weighted toward the interfaces
    (|y| large): a fraction `interface_frac` from the elements with the largest |y|,
    the rest uniformly. Returns torch tensors X (bfloat16 [S, n_in_pad]) and Y (float32 [S, npe]).
    """
    import torch

    rng = rng or np.random.default_rng(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    n_in_pad = (solver.closure_inputs + 15) // 16 * 16
    Xs, Ys = [], []
    solver.step(dt, first_step)
    for i in range(count):
        if i:
            solver.step(dt, every)
        X = torch.empty((solver.E, n_in_pad), dtype=torch.bfloat16, device=dev)
        Y = torch.empty((solver.E, solver.npe), dtype=torch.float32, device=dev)
        solver.closure_features(X)
        solver.closure_targets(Y)
        score = Y.abs().amax(dim=1).cpu().numpy()
        n = solver.E if max_per_snapshot is None else min(solver.E, max_per_snapshot)
        n_if = int(n * interface_frac)
        order = np.argsort(-score)
        pick = np.concatenate([order[:n_if], rng.choice(solver.E, n - n_if, replace=False)])
        idx = torch.from_numpy(np.unique(pick)).to(dev)
        Xs.append(X[idx])
        Ys.append(Y[idx])
    return torch.cat(Xs), torch.cat(Ys)


def train(mlp, X, Y, steps=2000, batch=4096, lr=2e-3, lr_min=2e-5, seed=0, log_every=0):
    """Adam on the mean squared error with a cosine learning-rate decay; returns the loss history
    (every `log_every` steps, plus the last)."""
    import torch

    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    S = X.shape[0]
    hist = []
    for it in range(steps):
        idx = torch.randint(0, S, (batch,), device=X.device, generator=g)
        xb, yb = X[idx].contiguous(), Y[idx].contiguous()
        lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / max(steps - 1, 1)))
        want = bool(log_every) and (it % log_every == 0 or it == steps - 1)
        loss = mlp.train_step(xb, yb, lr_t, want_loss=want or it == steps - 1)
        if loss is not None:
            hist.append((it, loss))
    return hist


def validation_error(mlp, X, Y):
    """Relative L2 error of the network on (X, Y): ||net(X) - Y|| / ||Y|| (in chunks of the
    network's inference capacity)."""
    import torch

    out = torch.empty_like(Y)
    for a in range(0, X.shape[0], mlp.max_rows):
        b = min(X.shape[0], a + mlp.max_rows)
        mlp.forward(X[a:b].contiguous(), out[a:b])
    torch.cuda.synchronize()
    return float(torch.linalg.norm(out - Y) / torch.linalg.norm(Y))
