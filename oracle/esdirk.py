"""TEST INFRASTRUCTURE ONLY: implicit time integration of the oracle's semi-discrete residual.

Sec. 3.1 (the time-integration paragraph) advances the DGSEM implicitly with the six-stage,
fourth-order explicit-first-stage singly diagonally implicit Runge-Kutta scheme of Kennedy and
Carpenter (2003): the implicit tableau of their ARK4(3)6L[2]SA, gamma = 1/4, stiffly accurate
(the last stage is the new solution), L-stable. The paper gives no solver details; this oracle
takes these readings (the GPU path takes the same ones):
  - each implicit stage G(X) = X - dt gamma R(X) - S_i = 0, S_i = U_n + dt sum_{j<i} a_ij R_j,
    is solved by Newton's method from the previous stage's value, stopping when
    ||G|| <= newton_tol ||S_i|| (Euclidean norms of the whole state);
  - the Newton systems (I - dt gamma J) d = -G are solved matrix-free (Jacobian-free
    Newton-Krylov): J v ~ (R(X + eps v) - R(X)) / eps, eps = sqrt(2^-52) (1 + ||X||) / ||v||,
    with restarted GMRES(m) (modified Gram-Schmidt, Givens rotations) to the relative residual
    krylov_tol, no preconditioner;
  - the stage derivative used by the later stages is R_i = (X_i - S_i) / (dt gamma), equal to
    R(X_i) at convergence, which saves one residual evaluation per stage.
Only tests/ (and the package smoke check / the benchmark's CPU legs) may use this module.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np

GAMMA = Fr(1, 4)
# ARK4(3)6L[2]SA, implicit part (Kennedy & Carpenter 2003): a_ij for j < i, diagonal gamma
A_EXACT = [
    [],
    [Fr(1, 4)],
    [Fr(8611, 62500), Fr(-1743, 31250)],
    [Fr(5012029, 34652500), Fr(-654441, 2922500), Fr(174375, 388108)],
    [Fr(15267082809, 155376265600), Fr(-71443401, 120774400), Fr(730878875, 902184768), Fr(2285395, 8070912)],
    [Fr(82889, 524892), Fr(0), Fr(15625, 83664), Fr(69875, 102672), Fr(-2260, 8211)],
]
STAGES = 6


def tableau(exact=False):
    """(A, b, c): the full 6x6 matrix with gamma on the diagonal from the second stage on, the
    weights (the last row: stiffly accurate) and the abscissae (row sums)."""
    z = Fr(0) if exact else 0.0
    conv = (lambda x: x) if exact else float
    A = [[z] * STAGES for _ in range(STAGES)]
    for i in range(1, STAGES):
        for j, a in enumerate(A_EXACT[i]):
            A[i][j] = conv(a)
        A[i][i] = conv(GAMMA)
    b = list(A[-1])
    c = [sum(row, z) for row in A]
    if not exact:
        return np.array(A), np.array(b), np.array(c)
    return A, b, c


def gmres(apply, rhs, tol, m, maxit):
    """Restarted GMRES(m) for apply(x) = rhs from x = 0; returns (x, iterations)."""
    n = rhs.size
    x = np.zeros(n)
    bn = float(np.linalg.norm(rhs))
    if bn == 0.0:
        return x, 0
    r = rhs.copy()
    its = 0
    while its < maxit:
        beta = float(np.linalg.norm(r))
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        k = 0
        for k in range(m):
            w = apply(V[k])
            its += 1
            for j in range(k + 1):  # modified Gram-Schmidt
                H[j, k] = float(w @ V[j])
                w = w - H[j, k] * V[j]
            H[k + 1, k] = float(np.linalg.norm(w))
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):  # earlier Givens rotations
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            d = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / d, H[k + 1, k] / d
            H[k, k], H[k + 1, k] = d, 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            if abs(g[k + 1]) <= tol * bn or its >= maxit:
                break
        kk = k + 1
        y = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
        x = x + V[:kk].T @ y
        if abs(g[kk]) <= tol * bn or its >= maxit:
            break
        r = rhs - apply(x)
    return x, its


def step(rhs, U, dt, newton_tol=1e-10, krylov_tol=1e-3, m=30, max_krylov=600, max_newton=20):
    """One ESDIRK4 step of U' = rhs(U); returns (U_new, stats) with stats = dict of Newton
    iterations, Krylov iterations and residual evaluations."""
    A, _, _ = tableau()
    g = float(GAMMA)
    shape = U.shape
    R = [rhs(U)]
    X = U.copy()
    st = {"newton": 0, "krylov": 0, "rhs": 1, "failed": 0}
    for i in range(1, STAGES):
        S = U + dt * sum(A[i, j] * R[j] for j in range(i))
        sn = float(np.linalg.norm(S))
        for it in range(max_newton + 1):
            RX = rhs(X)
            st["rhs"] += 1
            G = X - dt * g * RX - S
            if float(np.linalg.norm(G)) <= newton_tol * sn:
                break
            if it == max_newton:
                st["failed"] += 1
                break
            xn = float(np.linalg.norm(X))

            def apply(v):
                vn = float(np.linalg.norm(v))
                if vn == 0.0:
                    return np.zeros_like(v)
                eps = math.sqrt(2.0 ** -52) * (1.0 + xn) / vn
                Jv = (rhs(X + eps * v.reshape(shape)) - RX) / eps
                st["rhs"] += 1
                return v - dt * g * Jv.ravel()

            d, its = gmres(apply, -G.ravel(), krylov_tol, m, max_krylov)
            X = X + d.reshape(shape)
            st["newton"] += 1
            st["krylov"] += its
        R.append((X - S) / (dt * g))
    return X, st
