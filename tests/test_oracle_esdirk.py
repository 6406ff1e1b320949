"""Pins of the oracle's implicit time integration (oracle/esdirk.py: the six-stage fourth-order
ESDIRK of Sec. 3.1, Kennedy and Carpenter's ARK4(3)6L[2]SA implicit tableau, Jacobian-free
Newton-Krylov). No GPU.

Against facts independent of the code: the order conditions of the tableau in exact rational
arithmetic, the published abscissae, fourth-order convergence to closed-form ODE solutions,
L-stability, GMRES against a direct solve, and the closed-form uniform relaxation of the c
equation through the oracle's DG residual.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from oracle import esdirk as ES


def test_tableau_order_conditions_exact():
    A, b, c = ES.tableau(exact=True)
    n = ES.STAGES
    assert c == [Fr(0), Fr(1, 2), Fr(83, 250), Fr(31, 50), Fr(17, 20), Fr(1)]
    assert b == A[-1]  # stiffly accurate
    assert all(A[i][i] == Fr(1, 4) for i in range(1, n)) and A[0][0] == 0  # explicit first stage
    s = lambda f: sum(f(i) for i in range(n))  # noqa: E731
    Ac = [sum(A[i][j] * c[j] for j in range(n)) for i in range(n)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(n)) for i in range(n)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(n)) for i in range(n)]
    assert s(lambda i: b[i]) == 1
    assert s(lambda i: b[i] * c[i]) == Fr(1, 2)
    assert s(lambda i: b[i] * c[i] ** 2) == Fr(1, 3)
    assert s(lambda i: b[i] * Ac[i]) == Fr(1, 6)
    assert s(lambda i: b[i] * c[i] ** 3) == Fr(1, 4)
    assert s(lambda i: b[i] * c[i] * Ac[i]) == Fr(1, 8)
    assert s(lambda i: b[i] * Ac2[i]) == Fr(1, 12)
    assert s(lambda i: b[i] * AAc[i]) == Fr(1, 24)


def _run(rhs, y0, T, n):
    y = np.array([y0], dtype=float)
    for _ in range(n):
        y, _ = ES.step(rhs, y, T / n, newton_tol=1e-14, krylov_tol=1e-14, m=5)
    return y[0]


@pytest.mark.parametrize("rhs,exact", [
    (lambda y: -1.3 * y, lambda t: math.exp(-1.3 * t)),
    (lambda y: -y * y, lambda t: 1.0 / (1.0 + t)),
])
def test_fourth_order_convergence(rhs, exact):
    errs = [abs(_run(rhs, 1.0, 1.0, n) - exact(1.0)) for n in (8, 16, 32)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.7, (errs, rates)


def test_l_stability():
    """y' = lambda y with lambda dt = -1e8: the stiffly accurate, L-stable scheme damps the mode."""
    y = _run(lambda y: -1e8 * y, 1.0, 1.0, 1)
    assert abs(y) < 1e-6


def test_gmres_against_a_direct_solve():
    rng = np.random.Generator(np.random.PCG64(4))
    M = np.eye(40) * 3 + rng.standard_normal((40, 40)) * 0.2
    b = rng.standard_normal(40)
    x, its = ES.gmres(lambda v: M @ v, b, 1e-12, 15, 400)
    assert np.linalg.norm(M @ x - b) <= 1e-11 * np.linalg.norm(b)
    assert its > 15  # restarts happened


def test_uniform_relaxation_through_the_dg_residual():
    """Spatially constant rho, v = 0, c0 != rho: the residual reduces to the source, c(t) =
    rho + (c0 - rho) exp(-alpha t / beta). Steps of 5 beta/alpha (far above the explicit bound
    4.6 beta/alpha x cfl) converge at fourth order to the closed form."""
    o = O.Oracle(1, (4,), (0.0,), (1.0,), 3, O.NODES_GAUSS, alpha=100.0, beta=1e-3, kappa=1e-4, mu=1e-3)
    rho, c0 = 1.2, 1.25
    U = np.zeros(o.shape)
    U[0], U[2] = rho, c0
    lam = o.s.alpha / o.s.beta
    T = 20.0 / lam
    errs = []
    for n in (4, 8, 16):
        V = U.copy()
        for _ in range(n):
            V, st = ES.step(o.rhs, V, T / n, newton_tol=1e-13, krylov_tol=1e-12)
        assert st["failed"] == 0
        errs.append(np.abs(V[2] - (rho + (c0 - rho) * math.exp(-lam * T))).max())
        assert np.abs(V[0] - rho).max() < 1e-12
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.5, (errs, rates)


def _slab(E):
    o = O.Oracle(1, (E,), (0.0,), (1.0,), 3, O.NODES_GAUSS, alpha=100.0, beta=1e-2, kappa=1e-4, mu=1e-2)
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = 1.0 + 0.5 * np.tanh((0.25 - np.abs(x - 0.5)) / 0.05)
    U[1] = 0.05 * np.sin(2 * np.pi * x) * U[0]
    U[2] = U[0] * (1 + 0.01 * np.cos(2 * np.pi * x))
    return o, U


def test_coloured_block_jacobian_equals_the_dense_diagonal_blocks():
    """9 elements: 3 colours, three elements per colour, three apart (the closest that BR1's
    two-element reach allows). Perturbing them at once must give the same diagonal blocks as the
    dense forward-difference Jacobian built one unknown at a time."""
    o, U = _slab(9)
    assert ES.colours(9) == 3
    J = ES.block_jacobian(o.rhs, U, (9,))
    nvar, E, npe = U.shape
    n = nvar * npe
    R0 = o.rhs(U)
    for e in (0, 4, 8):
        for kk in range(n):
            v, node = divmod(kk, npe)
            W = U.copy()
            eps = math.sqrt(2.0 ** -52) * (1.0 + abs(U[v, e, node]))
            W[v, e, node] += eps
            col = ((o.rhs(W) - R0)[:, e, :]).reshape(n) / eps
            assert np.allclose(J[e, :, kk], col, rtol=1e-9, atol=1e-9 * np.abs(col).max())


def test_block_preconditioner_same_solution_fewer_krylov_iterations():
    o, U = _slab(20)
    dt = 100 * o.timestep(U, 0.5)
    U1, s1 = ES.step(o.rhs, U, dt, newton_tol=1e-11, krylov_tol=1e-6)
    U2, s2 = ES.step(o.rhs, U, dt, newton_tol=1e-11, krylov_tol=1e-6, nelem=(20,))
    assert s1["failed"] == 0 and s2["failed"] == 0
    assert np.abs(U1 - U2).max() <= 1e-8 * np.abs(U1).max()
    assert s2["krylov"] < s1["krylov"] / 2, (s1, s2)


def test_coloured_block_jacobian_2d_equals_the_dense_diagonal_blocks():
    """2D, 6 x 6 elements, N = 3 (64 unknowns per element): colours 3 x 3. Through BR1 an element's
    residual reaches every element within Manhattan distance two (its face neighbours' lifted
    gradients see their own face neighbours, diagonal ones included); same-coloured elements differ
    by at least three along some axis, so the coloured blocks equal the dense ones."""
    from paper_1912_12059_gb300 import inputs

    prm = dict(T=0.85, kappa=4e-3, alpha=1e3, beta=1e-3, mu=1e-2)
    ne = (6, 6)
    o = O.Oracle(2, ne, (0.0, 0.0), (1.0, 1.0), 3, O.NODES_GAUSS, **prm)
    U = np.asarray(inputs.droplets(o.coords(), [(0.5, 0.5)], [0.25], 0.3197, 1.8071, prm["kappa"]))
    J = ES.block_jacobian(o.rhs, U, ne)
    nvar, E, npe = U.shape
    n = nvar * npe
    R0 = o.rhs(U)
    for e in (0, 7, 20, 35):  # corners, interior, across the periodic wrap
        for kk in range(n):
            v, node = divmod(kk, npe)
            W = U.copy()
            eps = math.sqrt(2.0 ** -52) * (1.0 + abs(U[v, e, node]))
            W[v, e, node] += eps
            col = ((o.rhs(W) - R0)[:, e, :]).reshape(n) / eps
            assert np.allclose(J[e, :, kk], col, rtol=1e-9, atol=1e-9 * np.abs(col).max())


def test_gmres_terminates_after_as_many_iterations_as_distinct_eigenvalues():
    """For a diagonal (normal) matrix the Krylov space of any right-hand side has the dimension of
    the number of distinct eigenvalues, so GMRES reaches the exact solution in that many
    iterations: three here, out of a 30 x 30 system."""
    rng = np.random.Generator(np.random.PCG64(5))
    d = np.repeat([1.0, 2.0, 3.5], 10)
    b = rng.standard_normal(30)
    x, its = ES.gmres(lambda v: d * v, b, 1e-12, 20, 100)
    assert its == 3
    assert np.abs(d * x - b).max() < 1e-13


def test_step_statistics_of_a_scalar_linear_ode():
    """y' = -1.3 y, one unknown: every stage's Newton system is linear and one-dimensional, so
    one Newton iteration with one GMRES iteration solves it (to the forward difference's
    accuracy, within newton_tol = 1e-6); the residual evaluations are the first stage's, then per
    implicit stage the Newton residual, one Jacobian product and the converged check:
    1 + 5 x 3 = 16. A zero Newton limit stops all five stages at their initial iterate."""
    y = np.array([[1.0]])
    _, st = ES.step(lambda u: -1.3 * u, y, 0.1, newton_tol=1e-6, krylov_tol=1e-12)
    assert st == {"newton": 5, "krylov": 5, "rhs": 16, "failed": 0}
    _, st = ES.step(lambda u: -1.3 * u, y, 0.1, newton_tol=1e-6, krylov_tol=1e-12, max_newton=0)
    assert st == {"newton": 0, "krylov": 0, "rhs": 6, "failed": 5}
