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
    krylov_tol, without or with a right element-block preconditioner (the paper's code uses one;
    its construction is not given: here the inverses of the element blocks of I - dt gamma J(U_n),
    J's diagonal blocks from forward differences with an element colouring, once per step);
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


def colours(ne):
    """Colours per direction for the element-block Jacobian: with BR1 an element's residual depends
    on the states up to two elements away, so perturbing two elements of one colour leaves each
    one's residual to its own perturbation when they are at least three apart, across the periodic
    wrap too: the smallest divisor K >= 3 of ne (colour = coordinate mod K), else ne itself (every
    element its own colour)."""
    for K in range(3, ne + 1):
        if ne % K == 0:
            return K
    return ne


def block_jacobian(rhs, U, nelem):
    """Diagonal blocks dR_e/dU_e of the residual's Jacobian, [E][n][n] with n = nvar npe and the
    local unknown k = v npe + node, by forward differences: for each colour class and local unknown,
    every element of that class is perturbed at once, eps_e = sqrt(2^-52) (1 + |U_e,k|)."""
    nvar, E, npe = U.shape
    n = nvar * npe
    dim = len(nelem)
    K = [colours(ne) for ne in nelem]
    coord = np.zeros((E, dim), dtype=int)
    for e in range(E):
        r = e
        for k in range(dim):
            coord[e, k] = r % nelem[k]
            r //= nelem[k]
    col = np.zeros(E, dtype=int)
    stride = 1
    for k in range(dim):
        col += (coord[:, k] % K[k]) * stride
        stride *= K[k]
    R0 = rhs(U)
    J = np.zeros((E, n, n))
    for c in range(stride):
        members = np.nonzero(col == c)[0]
        if members.size == 0:
            continue
        for kk in range(n):
            v, node = divmod(kk, npe)
            W = U.copy()
            eps = math.sqrt(2.0 ** -52) * (1.0 + np.abs(U[v, members, node]))
            W[v, members, node] += eps
            dR = rhs(W) - R0
            for i, e in enumerate(members):
                J[e, :, kk] = dR[:, e, :].reshape(n) / eps[i]
    return J


def block_preconditioner(J, dtg):
    """Inverses of the element blocks of I - dt gamma J (right preconditioner of GMRES)."""
    n = J.shape[1]
    return np.linalg.inv(np.eye(n)[None] - dtg * J)


def apply_blocks(Minv, x, shape):
    """y_e = Minv_e x_e for the state-shaped vector x (flattened), [nvar][E][npe] layout."""
    nvar, E, npe = shape
    X = x.reshape(shape).transpose(1, 0, 2).reshape(E, nvar * npe)
    Y = np.einsum("eij,ej->ei", Minv, X)
    return Y.reshape(E, nvar, npe).transpose(1, 0, 2).reshape(-1)


def gmres(apply, rhs, tol, m, maxit, precond=None):
    """Restarted GMRES(m) for apply(x) = rhs from x = 0, right-preconditioned by precond (a map
    z -> M^-1 z, or None); returns (x, iterations)."""
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
            w = apply(V[k] if precond is None else precond(V[k]))
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
        x = x + (V[:kk].T @ y if precond is None else precond(V[:kk].T @ y))
        if abs(g[kk]) <= tol * bn or its >= maxit:
            break
        r = rhs - apply(x)
    return x, its


def step(rhs, U, dt, newton_tol=1e-10, krylov_tol=1e-3, m=30, max_krylov=600, max_newton=20, nelem=None):
    """One ESDIRK4 step of U' = rhs(U); returns (U_new, stats) with stats = dict of Newton
    iterations, Krylov iterations and residual evaluations. nelem (elements per direction) turns
    on the element-block preconditioner: the blocks of I - dt gamma J(U_n), built once per step
    by coloured forward differences (their residual evaluations are counted)."""
    A, _, _ = tableau()
    g = float(GAMMA)
    shape = U.shape
    R = [rhs(U)]
    X = U.copy()
    st = {"newton": 0, "krylov": 0, "rhs": 1, "failed": 0}
    precond = None
    if nelem is not None:
        J = block_jacobian(rhs, U, nelem)
        K = 1
        for ne in nelem:
            K *= colours(ne)
        st["rhs"] += 1 + K * shape[0] * shape[2]
        Minv = block_preconditioner(J, dt * g)
        precond = lambda z: apply_blocks(Minv, z, shape)  # noqa: E731
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

            d, its = gmres(apply, -G.ravel(), krylov_tol, m, max_krylov, precond)
            X = X + d.reshape(shape)
            st["newton"] += 1
            st["krylov"] += its
        R.append((X - S) / (dt * g))
    return X, st
