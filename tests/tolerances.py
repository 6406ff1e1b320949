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


def state_rel_err(Ug, Uo):
    """Relative L-infinity error of a state, each variable against its own scale:
    max over v of max|Ug[v] - Uo[v]| / max|Uo[v]|, so that a small variable (momentum of a
    fluid nearly at rest next to rho and c of order one) is held to its own size. A variable
    that is identically zero in the oracle's state is measured against the largest variable's
    scale. Returns (the maximum, the per-variable list)."""
    big = float(np.abs(Uo).max())
    errs = []
    for v in range(Uo.shape[0]):
        sc = float(np.abs(Uo[v]).max())
        errs.append(float(np.abs(Ug[v] - Uo[v]).max()) / (sc if sc > 0.0 else max(big, 1e-300)))
    return max(errs), errs
