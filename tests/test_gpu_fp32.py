"""FP32 operator (NSK_FP32_MIXED): the DG operator in FP32 with the equation of
state, wave speeds, time step and diagnostic sums in FP64.

Single-operator bound: the FP64 bound of the parity tests scaled from the FP64
to the FP32 unit roundoff (about 1e-6 of (2/h)(N+1)^2 max|flux|, plus 1e-5 of
the residual). Over time the FP32 operator's acceptance is the density L2 error
relative to the FP64 run, required <= 1e-4; it is measured here on small
droplet problems and reported by the benchmark at full size.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu


def _solver(dim, ne, N, precision, **prm):
    p = dict(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3)
    p.update(prm)
    s = nsk.Solver(dim, ne, N, [0.0] * dim, [1.0] * dim, 0, precision)
    s.set_params(**p)
    return s, p


@pytest.mark.parametrize("flux", [nsk.NSK_FLUX_LF, nsk.NSK_FLUX_HLLC])
@pytest.mark.parametrize("dim,ne,N", [(1, (40,), 3), (2, (7, 6), 4), (3, (5, 4, 3), 3)])
def test_fp32_rhs_within_fp32_bound(gpu, dim, ne, N, flux):
    from tolerances import rhs_tolerance

    s, p = _solver(dim, ne, N, nsk.NSK_FP32_MIXED, mu=2e-2, kappa=1e-3)
    s.set_flux(flux)
    o = O.Oracle(dim, ne, [0.0] * dim, [1.0] * dim, N, 0, flux=flux, **p)
    U = inputs.random_state(o.shape, seed=50 + dim)
    U32 = U.astype(np.float32).astype(np.float64)  # the FP32 context stores the state in FP32
    s.set_state(U)
    Rg = s.rhs()
    Ro = o.rhs(U32)
    tol64 = rhs_tolerance(o, U32, Ro)
    for v in range(o.nvar):
        tol = tol64[v] * (2.0**-24 / 2.0**-53) * 0.5 + 1e-5 * np.abs(Ro[v]).max()
        err = float(np.abs(Rg[v] - Ro[v]).max())
        assert err <= tol, (v, err, tol)
    s.close()


def _density_l2_rel(a, b):
    return float(np.sqrt(((a[0] - b[0]) ** 2).sum() / (b[0] ** 2).sum()))


@pytest.mark.parametrize("case", ["droplets2d", "collision3d"])
def test_fp32_density_error_vs_fp64(gpu, case):
    rv, rl, _ = O.maxwell(0.85)
    if case == "droplets2d":
        dim, ne, N, prm = 2, (24, 24), 4, dict(mu=2e-3, alpha=1e3)
        s64, p = _solver(dim, ne, N, nsk.NSK_FP64, **prm)
        U = inputs.droplets(s64.node_coords(), ((0.35, 0.5), (0.65, 0.5)), (0.15, 0.12), rv, rl, 1e-4)
        U = inputs.add_density_noise(U, 1e-4)
    else:
        dim, ne, N, prm = 3, (12, 12, 12), 3, {}
        s64, p = _solver(dim, ne, N, nsk.NSK_FP64, **prm)
        v = inputs.collision_velocity(40.0, 0.2, 1e-4, rv, rl)
        U = inputs.head_on_collision(s64.node_coords(), v, 0.2, rho_vap=rv, rho_liq=rl, kappa=1e-4)
    s32, _ = _solver(dim, ne, N, nsk.NSK_FP32_MIXED, **prm)
    s64.set_state(U)
    s32.set_state(U)
    dt = s64.compute_dt(0.5)
    assert abs(s32.compute_dt(0.5) - dt) <= 1e-6 * dt
    s64.step(dt, 200)
    s32.step(dt, 200)
    U64, U32 = s64.get_state(), s32.get_state()
    err = _density_l2_rel(U32, U64)
    m64, _, _ = s64.diagnostics()
    m32, _, _ = s32.diagnostics()
    print(f"{case}: FP32 density L2 rel error after 200 steps {err:.3e}, mass drift {abs(m32 - m64) / m64:.2e}")
    assert err <= 1e-4
    assert abs(m32 - m64) <= 1e-6 * m64
    s64.close()
    s32.close()


def test_line_schedule_at_full_size(gpu):
    """The benchmark's FP32 configuration, the 64^3 head-on collision (N = 3, We = 40), under the
    line-per-thread kernels the autotuner picks there (schedule 128,4) against the separate face
    pass with node-per-thread kernels (256,0): residual and three steps equal bit for bit, and the
    density after the steps within the FP32 bound of the FP64 run."""
    wl = inputs.head_on_collision_3d(we=40.0, nelem=64)
    out = {}
    for prec, sched in ((nsk.NSK_FP32_MIXED, (256, 0)), (nsk.NSK_FP32_MIXED, (128, 4)), (nsk.NSK_FP64, (256, 0))):
        s = nsk.Solver(3, wl.nelem, 3, [0, 0, 0], [1, 1, 1], 0, prec)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        s.set_schedule(*sched)
        s.set_state(wl.initial_state(s.node_coords()))
        R = s.rhs() if prec == nsk.NSK_FP32_MIXED else None
        s.step(2.3e-6, 3)
        out[(prec, sched)] = (R, s.get_state())
        s.close()
    a, b = out[(nsk.NSK_FP32_MIXED, (256, 0))], out[(nsk.NSK_FP32_MIXED, (128, 4))]
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert _density_l2_rel(b[1], out[(nsk.NSK_FP64, (256, 0))][1]) <= 1e-5
