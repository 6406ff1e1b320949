"""Design order of the oracle on manufactured solutions (no GPU).

A smooth periodic single-phase solution (rho in the convex range around 2.1)
is manufactured with sympy: the source S_mms = U_t + div(F^c - F^v) - S of
model II (Eq. fluxes_sources_model2) is derived symbolically, added to the
oracle's semi-discrete residual, and the system is advanced with the oracle's
own five-stage RK4 coefficients. The L2 error at the final time must fall at
the DGSEM design rate (about N+1) under mesh refinement; a dropped or
mis-signed flux or source term, or a wrong metric factor, leaves an O(1)
error that does not converge.
"""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

import oracle as O  # noqa: E402

T, KAPPA, ALPHA, BETA, MU = 0.85, 1e-2, 1.0, 1.0, 1e-2


def _model_terms(dim, rho, vel, c, X, t):
    """U, F^c_k - F^v_k and the model source S as sympy expressions."""
    p_alpha = 8 * T * rho / (3 - rho) - 3 * rho**2 + ALPHA * rho**2 / 2
    grad = lambda f: [sympy.diff(f, X[k]) for k in range(dim)]  # noqa: E731
    gv = [grad(vel[a]) for a in range(dim)]  # gv[a][k] = d v_a / d x_k
    div = sum(gv[a][a] for a in range(dim))
    gc = grad(c)
    U = [rho] + [rho * vel[a] for a in range(dim)] + [c]
    fluxes = []
    for k in range(dim):
        f = [rho * vel[k]]
        for a in range(dim):
            tau = MU * (gv[a][k] + gv[k][a] - (sympy.Rational(2, 3) * div if a == k else 0))
            f.append(rho * vel[k] * vel[a] + (p_alpha if a == k else 0) - tau)
        f.append(-KAPPA / BETA * gc[k])
        fluxes.append(f)
    S = [0] + [ALPHA * rho * gc[a] for a in range(dim)] + [ALPHA / BETA * (rho - c)]
    return U, fluxes, S


def _manufactured(dim):
    t = sympy.Symbol("t")
    X = sympy.symbols("x0:%d" % dim)
    tp = 2 * sympy.pi
    if dim == 1:
        x = X[0]
        rho = 2.1 + 0.1 * sympy.sin(tp * (x - t))
        vel = [0.3 + 0.1 * sympy.sin(tp * (x + t))]
        c = rho + 0.01 * sympy.cos(tp * (x - 2 * t))
    else:
        x, y = X
        rho = 2.1 + 0.05 * sympy.sin(tp * (x - t)) * sympy.cos(tp * y) + 0.03 * sympy.sin(tp * y + 1)
        vel = [0.2 + 0.1 * sympy.sin(tp * (x + y - t)), -0.1 + 0.08 * sympy.cos(tp * (x - 2 * y) + t)]
        c = rho + 0.01 * sympy.sin(tp * (x + y) - t)
    U, F, S = _model_terms(dim, rho, vel, c, X, t)
    nv = dim + 2
    src = []
    for v in range(nv):
        expr = sympy.diff(U[v], t) + sum(sympy.diff(F[k][v], X[k]) for k in range(dim)) - S[v]
        src.append(sympy.lambdify((t, *X), expr, "numpy"))
    exact = [sympy.lambdify((t, *X), U[v], "numpy") for v in range(nv)]
    return exact, src


def _evaluate(funcs, t, x):
    out = np.empty((len(funcs),) + x.shape[1:])
    for v, f in enumerate(funcs):
        out[v] = np.broadcast_to(f(t, *x), x.shape[1:])
    return out


def _run(dim, ne, N, tend, exact, src, flux=O.FLUX_LF):
    orc = O.Oracle(dim, (ne,) * dim, (0.0,) * dim, (1.0,) * dim, N, O.NODES_GAUSS, T=T, kappa=KAPPA,
                   alpha=ALPHA, beta=BETA, mu=MU, flux=flux)
    x = orc.coords()
    U = _evaluate(exact, 0.0, x)
    A, B, Cc = O.lsrk4_coeffs()
    dt0 = 0.3 * orc.timestep(U, 1.0)
    nsteps = int(math.ceil(tend / dt0))
    dt = tend / nsteps
    K = np.zeros_like(U)
    t = 0.0
    for _ in range(nsteps):
        for s in range(5):
            R = orc.rhs(U) + _evaluate(src, t + Cc[s] * dt, x)
            K = A[s] * K + dt * R
            U = U + B[s] * K
        t += dt
    err = U - _evaluate(exact, tend, x)
    h = 1.0 / ne
    wq = np.ones(orc.npe)
    for n in range(orc.npe):
        r = n
        for k in range(dim):
            wq[n] *= orc.w[r % orc.np] * h / 2
            r //= orc.np
    return math.sqrt(float((err[0] ** 2 * wq).sum()))


@pytest.mark.parametrize("dim,N,meshes,tend", [
    (1, 2, (4, 8, 16), 0.1),
    (1, 3, (4, 8, 16), 0.1),
    (2, 2, (4, 8), 0.05),
    (2, 3, (4, 8), 0.05),
])
def test_design_order(dim, N, meshes, tend):
    exact, src = _manufactured(dim)
    errs = [_run(dim, ne, N, tend, exact, src) for ne in meshes]
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(meshes[i + 1] / meshes[i]) for i in range(len(errs) - 1)]
    print(dim, N, errs, rates)
    assert errs[-1] < 1e-3
    assert min(rates) > N + 0.5, (errs, rates)


@pytest.mark.parametrize("dim,N,meshes,tend", [
    (1, 3, (4, 8, 16), 0.1),
    (2, 2, (4, 8), 0.05),
])
def test_design_order_hllc(dim, N, meshes, tend):
    """The same manufactured solution with the HLLC face flux."""
    exact, src = _manufactured(dim)
    errs = [_run(dim, ne, N, tend, exact, src, flux=O.FLUX_HLLC) for ne in meshes]
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(meshes[i + 1] / meshes[i]) for i in range(len(errs) - 1)]
    print(dim, N, errs, rates)
    assert errs[-1] < 1e-3
    assert min(rates) > N + 0.5, (errs, rates)
