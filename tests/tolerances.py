"""Parity tolerances shared by the GPU tests (derived from the arithmetic of the residual)."""
import numpy as np


def rhs_tolerance(o, U, R):
    """Per-variable bound on |R_gpu - R_orc| derived from the arithmetic: the residual is a
    sum of flux differences scaled by 2/h and the derivative matrix, so rounding in either
    evaluation is a few ulps of rh * (N+1)^2 * max|flux| (the largest term that cancels),
    plus 1e-12 of the residual itself. Fluxes: rho -> |m|; momentum -> |m m / rho| + |p_alpha|;
    c -> (kappa/beta) |grad c|."""
    d = o.dim
    s = o.s
    rh = max(2.0 * o.nelem[k] / (o.hi[k] - o.lo[k]) for k in range(d))
    rho = U[0]
    mom = U[1:1 + d]
    pa = 8 * s.T * rho / (3 - rho) - 3 * rho**2 + 0.5 * s.alpha * rho**2
    Q = o.lift(U)
    gc = max(np.abs(Q[k * (d + 1) + d]).max() for k in range(d))
    F = [np.abs(mom).max()]
    F += [float((np.abs(mom) * np.abs(mom[a]) / rho).max() + np.abs(pa).max()) for a in range(d)]
    F += [s.kappa / s.beta * gc]
    amp = rh * (o.np ** 2)
    return [1e-12 * np.abs(R[v]).max() + 2e-15 * amp * F[v] for v in range(o.nvar)]
