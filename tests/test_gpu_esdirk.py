"""Implicit time integration on the GPU (nsk_step_esdirk: the six-stage fourth-order ESDIRK of
Sec. 3.1 with Jacobian-free Newton-Krylov) against the oracle's ESDIRK (oracle/esdirk.py).

Both solve every implicit stage to the same Newton tolerance with the same algorithm; the Krylov
iterates differ by rounding (dot products in another order), so the stage solutions agree to
the Newton tolerance times the conditioning, not bit for bit: relative L-infinity <= 1e-8 with
newton_tol = 1e-11 and krylov_tol = 1e-8 below. The uniform relaxation has a closed form.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import esdirk as ES
from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu

NT, KT = 1e-11, 1e-8


def pair(dim, ne, N, **prm):
    s = nsk.Solver(dim, ne, N, [0.0] * dim, [1.0] * dim, 0, nsk.NSK_FP64)
    s.set_params(**prm)
    o = O.Oracle(dim, ne, (0.0,) * dim, (1.0,) * dim, N, O.NODES_GAUSS, **prm)
    return s, o


def test_uniform_relaxation_closed_form(gpu):
    prm = dict(T=0.85, kappa=1e-4, alpha=100.0, beta=1e-3, mu=1e-3)
    s, o = pair(1, (4,), 3, **prm)
    rho, c0 = 1.2, 1.25
    U = np.zeros(o.shape)
    U[0], U[2] = rho, c0
    s.set_state(U)
    lam = prm["alpha"] / prm["beta"]
    T, n = 20.0 / lam, 8
    st = s.step_esdirk(T / n, n, newton_tol=1e-13, krylov_tol=1e-12)
    Ug = s.get_state()
    assert st["failed"] == 0
    exact = rho + (c0 - rho) * math.exp(-lam * T)
    V = U.copy()
    for _ in range(n):
        V, _ = ES.step(o.rhs, V, T / n, newton_tol=1e-13, krylov_tol=1e-12)
    assert np.abs(Ug[2] - V[2]).max() < 1e-12
    assert np.abs(Ug[2] - exact).max() < 2e-6
    s.close()


@pytest.mark.parametrize("fac", [10.0, 100.0])
def test_parity_1d_interface(gpu, fac):
    """The 1D static phase interface (alpha = 100, beta = 1e-2), one step at fac times the
    explicit CFL-0.5 step."""
    prm = dict(T=0.85, kappa=1e-4, alpha=100.0, beta=1e-2, mu=1e-2)
    s, o = pair(1, (16,), 3, **prm)
    rv, rl, _ = O.maxwell(0.85)
    U = inputs.slab_1d(o.coords(), rv, rl, 1e-4)
    dt = fac * o.timestep(U, 0.5)
    s.set_state(U)
    st = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT)
    Ug = s.get_state()
    Uo, sto = ES.step(o.rhs, U, dt, newton_tol=NT, krylov_tol=KT)
    assert st["failed"] == 0 and sto["failed"] == 0
    for v in range(o.nvar):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-8 * np.abs(Uo[v]).max() + 1e-12, v
    assert abs(st["newton"] - sto["newton"]) <= 2
    s.close()


def test_parity_3d_collision(gpu):
    prm = dict(T=0.85, kappa=4e-3, alpha=1e3, beta=1e-3, mu=1e-2)
    s, o = pair(3, (4, 4, 3), 2, **prm)
    x = o.coords()
    U = inputs.head_on_collision(x, 0.3, radius=0.25, rho_vap=0.3197, rho_liq=1.8071, kappa=prm["kappa"])
    dt = 5.0 * o.timestep(U, 0.5)
    s.set_state(U)
    st = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT)
    Ug = s.get_state()
    Uo, sto = ES.step(o.rhs, U, dt, newton_tol=NT, krylov_tol=KT)
    assert st["failed"] == 0 and sto["failed"] == 0
    for v in range(o.nvar):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-8 * np.abs(Uo[v]).max() + 1e-12, v
    s.close()


def test_esdirk_argument_checks(gpu):
    s = nsk.Solver(1, (8,), 3, [0.0], [1.0], 0, nsk.NSK_FP32_MIXED)
    s.set_params()
    s.set_state(inputs.random_state(s.shape, seed=1))
    with pytest.raises(RuntimeError):
        s.step_esdirk(1e-5, 1)
    s.close()
    s = nsk.Solver(1, (8,), 3, [0.0], [1.0], 0, nsk.NSK_FP64)
    s.set_params()
    with pytest.raises(RuntimeError):
        s.step_esdirk(1e-5, 1)  # no state yet
    s.set_state(inputs.random_state(s.shape, seed=1))
    with pytest.raises(RuntimeError):
        s.step_esdirk(-1e-5, 1)
    with pytest.raises(RuntimeError):
        s.step_esdirk(1e-5, 1, krylov_dim=0)
    s.close()


@pytest.mark.parametrize("E", [16, 7])
def test_parity_block_preconditioned(gpu, E):
    """The element-block preconditioner (colours: 4 for 16 elements, every element its own for 7):
    the 1D interface at 100x the explicit step against the oracle's preconditioned step."""
    prm = dict(T=0.85, kappa=1e-4, alpha=100.0, beta=1e-2, mu=1e-2)
    s, o = pair(1, (E,), 3, **prm)
    rv, rl, _ = O.maxwell(0.85)
    U = inputs.slab_1d(o.coords(), rv, rl, 1e-4)
    dt = 100.0 * o.timestep(U, 0.5)
    s.set_state(U)
    st = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT, block_precond=True)
    Ug = s.get_state()
    Uo, sto = ES.step(o.rhs, U, dt, newton_tol=NT, krylov_tol=KT, nelem=(E,))
    assert st["failed"] == 0 and sto["failed"] == 0
    for v in range(o.nvar):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-8 * np.abs(Uo[v]).max() + 1e-12, v
    s.set_state(U)
    plain = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT)
    assert st["krylov"] < plain["krylov"]
    s.close()


def test_parity_stiff_paper_parameters(gpu):
    """The paper's alpha = 1e3, beta = 1e-3, mu = 1e-3 (the explicit step bound by the c equation's
    source): one preconditioned step of 1000x the explicit CFL-0.5 step on the 1D interface
    against the oracle's, and fewer Krylov iterations than without the preconditioner."""
    prm = dict(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3)
    s, o = pair(1, (16,), 3, **prm)
    rv, rl, _ = O.maxwell(0.85)
    U = inputs.slab_1d(o.coords(), rv, rl, 1e-4)
    dt = 1000.0 * o.timestep(U, 0.5)
    s.set_state(U)
    st = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT, block_precond=True)
    Ug = s.get_state()
    Uo, sto = ES.step(o.rhs, U, dt, newton_tol=NT, krylov_tol=KT, nelem=(16,))
    assert st["failed"] == 0 and sto["failed"] == 0
    for v in range(o.nvar):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-8 * np.abs(Uo[v]).max() + 1e-12, v
    s.set_state(U)
    plain = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT)
    assert plain["failed"] == 0 and st["krylov"] < plain["krylov"] / 2
    s.close()


def test_parity_block_preconditioned_2d(gpu):
    """2D, 6 x 6 elements, N = 3: 64-unknown blocks (the inversion's 64 KB of dynamic shared
    memory), 3 x 3 colours; a droplet at 100x the explicit step against the oracle's
    preconditioned step, with fewer Krylov iterations than without the preconditioner."""
    prm = dict(T=0.85, kappa=4e-3, alpha=1e3, beta=1e-3, mu=1e-2)
    s, o = pair(2, (6, 6), 3, **prm)
    U = np.asarray(inputs.droplets(o.coords(), [(0.5, 0.5)], [0.25], 0.3197, 1.8071, prm["kappa"]))
    dt = 100.0 * o.timestep(U, 0.5)
    s.set_state(U)
    st = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT, block_precond=True)
    Ug = s.get_state()
    Uo, sto = ES.step(o.rhs, U, dt, newton_tol=NT, krylov_tol=KT, nelem=(6, 6))
    assert st["failed"] == 0 and sto["failed"] == 0
    for v in range(o.nvar):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-8 * np.abs(Uo[v]).max() + 1e-12, v
    s.set_state(U)
    plain = s.step_esdirk(dt, 1, newton_tol=NT, krylov_tol=KT)
    assert st["krylov"] < plain["krylov"]
    s.close()


def test_block_preconditioner_size_limit(gpu):
    """Blocks above 64 unknowns (2D, N = 4: 4 x 25) are rejected; N = 3 is accepted."""
    s = nsk.Solver(2, (3, 3), 4, [0.0, 0.0], [1.0, 1.0], 0, nsk.NSK_FP64)
    s.set_params()
    s.set_state(inputs.random_state(s.shape, seed=2))
    with pytest.raises(RuntimeError):
        s.step_esdirk(1e-6, 1, block_precond=True)
    s.close()
