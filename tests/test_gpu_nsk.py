"""The original NSK equations on the GPU (nsk_set_model(NSK_MODEL_NSK), FP64) against the
oracle's original NSK path.

Residual tolerance, per variable: the residual sums flux differences scaled by 2/h and the
derivative matrix, so rounding is a few ulps of (2/h)(N+1)^2 times the largest flux that
cancels: mass |m|; momentum |m m/rho| + |p| + kappa (rho |lap rho| + 3/2 |grad rho|^2), and
lap rho itself comes out of a second lifting, whose rounding is relative to (2/h)(N+1)^2
|grad rho|. After 100 LSRK4 steps the relative L-infinity error must be <= 1e-11, as for
model II.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs, nsk
from tolerances import state_rel_err

pytestmark = pytest.mark.gpu


def make_pair(dim, ne, N, nt=0, hi=None, **prm):
    p = dict(T=0.85, kappa=1e-3, alpha=1e3, beta=1e-3, mu=2e-2)
    p.update(prm)
    hi = hi or [1.0] * dim
    s = nsk.Solver(dim, ne, N, [0.0] * dim, hi, nt, nsk.NSK_FP64)
    s.set_params(**p)
    s.set_model(nsk.NSK_MODEL_NSK)
    o = O.Oracle(dim, ne, [0.0] * dim, hi, N, nt, model=O.MODEL_NSK, **p)
    return s, o


def tolerance(o, U, R):
    d, s = o.dim, o.s
    rh = max(2.0 * o.nelem[k] / (o.hi[k] - o.lo[k]) for k in range(d))
    amp = rh * o.np**2
    rho, mom = U[0], U[1:1 + d]
    p = 8 * s.T * rho / (3 - rho) - 3 * rho**2
    Q = o.lift(U)
    g = np.sqrt(sum(Q[k * (d + 1) + d] ** 2 for k in range(d)))
    lap = o.lift2(U)
    kort = s.kappa * (rho * (np.abs(lap) + amp * g) + 1.5 * g * g)
    F = [np.abs(mom).max()]
    F += [float((np.abs(mom) * np.abs(mom[a]) / rho + np.abs(p) + kort).max()) for a in range(d)]
    return [1e-12 * np.abs(R[v]).max() + 2e-15 * amp * F[v] for v in range(d + 1)]


CASES = [(1, (40,), 3, 0), (1, (13,), 4, 1), (2, (7, 5), 4, 0), (2, (6, 6), 2, 1), (3, (5, 3, 3), 3, 0),
         (3, (3, 3, 2), 4, 0), (3, (2, 3, 2), 5, 0)]


@pytest.mark.parametrize("dim,ne,N,nt", CASES)
def test_rhs_and_lift_parity(gpu, dim, ne, N, nt):
    s, o = make_pair(dim, ne, N, nt, hi=[1.0, 0.8, 1.3][:dim])
    U = inputs.random_state((dim + 2,) + o.shape[1:], seed=400 + dim * 10 + N)[:dim + 1]
    s.set_state(U)
    Qg, Qo = s.lift(), o.lift(U)
    for c in range(o.nq):
        assert np.abs(Qg[c] - Qo[c]).max() <= 1e-12 * (np.abs(Qo[c]).max() + 1e-3 * np.abs(Qo).max()), c
    Rg, Ro = s.rhs(), o.rhs(U)
    tol = tolerance(o, U, Ro)
    for v in range(o.nvar):
        err = np.abs(Rg[v] - Ro[v]).max()
        assert err <= tol[v], (v, err, tol[v])
    s.close()


def test_free_stream(gpu):
    s, o = make_pair(3, (4, 3, 5), 3, hi=[1.0, 0.7, 1.3])
    U = np.zeros(o.shape)
    U[0], U[1], U[2], U[3] = 1.3, 0.52, 0.13, -0.26
    s.set_state(U)
    assert np.abs(s.rhs()).max() < 1e-9
    s.close()


def _case(name):
    rv, rl, _ = O.maxwell(0.85)
    if name == "slab1d":
        s, o = make_pair(1, (64,), 3, mu=1e-2, kappa=4e-4)
        U = inputs.slab_1d(o.coords(), rv, rl, 4e-4)[:2]
    elif name == "droplets2d":
        s, o = make_pair(2, (16, 16), 4, mu=2e-3, kappa=1e-3)
        U = inputs.droplets(o.coords(), ((0.35, 0.5), (0.65, 0.5)), (0.15, 0.12), rv, rl, 1e-3)
        U = inputs.add_density_noise(U, 1e-4)[:3]
    else:
        s, o = make_pair(3, (7, 6, 5), 3, mu=1e-2, kappa=4e-3)
        v = inputs.collision_velocity(40.0, 0.2, 4e-3, rv, rl)
        U = inputs.head_on_collision(o.coords(), v, 0.2, rho_vap=rv, rho_liq=rl, kappa=4e-3)[:4]
    return s, o, U


@pytest.mark.parametrize("name", ["slab1d", "droplets2d", "collision3d"])
def test_step_parity_100(gpu, name):
    s, o, U = _case(name)
    dt = o.timestep(U, 0.5)
    s.set_state(U)
    assert abs(s.compute_dt(0.5) - dt) <= 1e-13 * dt
    s.step(dt, 100)
    Ug = s.get_state()
    Uo = o.step(U, dt, 100)
    err, per_var = state_rel_err(Ug, Uo)  # each variable against its own scale
    assert err <= 1e-11, per_var
    mg, eg, lg = s.diagnostics()
    mo, eo, lo_ = o.diagnostics(Uo)
    assert abs(mg - mo) <= 1e-12 * abs(mo)
    assert abs(eg - eo) <= 1e-10 * abs(eo)
    assert lg == 0.0 and lo_ == 0.0
    s.close()


def test_adaptive_step_and_call_order(gpu):
    s, o, U = _case("slab1d")
    s.set_state(U)
    s.step(-0.5, 3)
    Uo = U
    for _ in range(3):
        Uo = o.step(Uo, o.timestep(Uo, 0.5), 1)
    assert float(np.abs(s.get_state() - Uo).max() / np.abs(Uo).max()) < 1e-12
    s.set_model(nsk.NSK_MODEL_RELAXATION)  # switching the model needs a new state
    with pytest.raises(nsk.NskError) as ei:
        s.rhs()
    assert ei.value.code == nsk.NSK_ERR_STATE
    s.close()
    f32 = nsk.Solver(1, (8,), 3, [0.0], [1.0], 0, nsk.NSK_FP32_MIXED)
    f32.set_params(T=0.85, kappa=1e-3, alpha=1e3, beta=1e-3, mu=1e-2)
    with pytest.raises(nsk.NskError) as ei:
        f32.set_model(nsk.NSK_MODEL_NSK)  # FP64 only
    assert ei.value.code == nsk.NSK_ERR_ARG
    f32.close()
