"""Finite-volume sub-cell shock capturing and Dirichlet boundaries on the GPU (1D, FP64, model
II: nsk_set_subcell, nsk_set_dirichlet) against the oracle's sub-cell path.

Residual tolerance: both sides evaluate the same arithmetic in FP64 in different orders, so the
residual differs by a few ulps of its largest cancelling terms: the flux differences amplified
by the DG derivative (2/h)(N+1)^2 (the FV difference quotient 1/dx = (N+1)/h is smaller) and the
stiff source (alpha/beta) rho. The bound below takes 1e-13 of that scale. Indicator decisions
are integers decided in FP64 on both sides; the test states keep every indicator away from the
thresholds, and the flags must then agree exactly. After 100 steps of the Riemann problem the
relative L-infinity error must be <= 1e-10.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu

PRM = dict(T=0.85, kappa=1e-6, alpha=100.0, beta=1e-3, mu=1e-3)
LEFT, RIGHT = (2.0, 0.0, 2.0), (0.1, 0.0, 0.1)


def make_pair(E, N, dirichlet, flux=nsk.NSK_FLUX_HLLC, subcell=True, **prm):
    p = dict(PRM)
    p.update(prm)
    s = nsk.Solver(1, (E,), N, [0.0], [1.0], 0, nsk.NSK_FP64)
    s.set_params(**p)
    s.set_flux(flux)
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, O.NODES_GAUSS, flux=flux, **p)
    if subcell:
        s.set_subcell(True, -6.0, -8.0)
    if dirichlet:
        s.set_dirichlet(LEFT, RIGHT)
    o.fv_setup(dirichlet=dirichlet, Ub_lo=LEFT, Ub_hi=RIGHT, ind_upper=-6.0, ind_lower=-8.0)
    return s, o


def scale(o, U, N, E):
    rho, m, c = U[0], U[1], U[2]
    pa = 8 * o.s.T * rho / (3 - rho) - 3 * rho**2 + o.s.alpha * rho**2 / 2
    amp = 2.0 * E * (N + 1) ** 2
    flux = np.abs(m).max() + np.abs(m * m / rho).max() + np.abs(pa).max()
    diff = o.s.kappa / o.s.beta * amp * np.abs(c).max() + o.s.mu * amp * np.abs(m / rho).max()
    return amp * (flux + diff) + o.s.alpha / o.s.beta * rho.max() + o.s.alpha * rho.max() * amp * np.abs(c).max()


def mixed_state(o, seed):
    """A Riemann-like state with random perturbations (in range for both representations)."""
    x = o.coords()
    U = inputs.riemann_1d(x, 1.8, 0.3, 0.43)
    R = inputs.random_state(o.shape, seed=seed, rho_range=(0.9, 1.1), v_amp=0.1, c_amp=0.02)
    U[0] *= R[0]
    U[1] = U[0] * (R[1] / R[0])
    U[2] = U[0] * (R[2] / R[0])
    return U


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("E", [1, 3, 17])
@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("flux", [nsk.NSK_FLUX_LF, nsk.NSK_FLUX_HLLC])
def test_fv_rhs_parity(gpu, N, E, dirichlet, flux):
    s, o = make_pair(E, N, dirichlet, flux)
    U = mixed_state(o, 11 * N + E)
    flags = (np.random.Generator(np.random.PCG64(E + 7 * N)).uniform(size=E) < 0.5).astype(np.int32)
    s.set_state(U)
    s.set_subcell_flags(flags)
    Rg, Ro = s.rhs(), o.fv_rhs(U, flags)
    assert np.abs(Rg - Ro).max() <= 1e-13 * scale(o, U, N, E)
    s.close()


@pytest.mark.parametrize("N", [2, 3])
def test_all_dg_periodic_equals_the_dg_path(gpu, N):
    """With every element DG and periodic boundaries the sub-cell path's residual is the DG
    residual of the ordinary stage kernels."""
    E = 16
    s, o = make_pair(E, N, dirichlet=False)
    U = inputs.random_state(o.shape, seed=3)
    s.set_state(U)
    R_fv = s.rhs()
    s2 = nsk.Solver(1, (E,), N, [0.0], [1.0], 0, nsk.NSK_FP64)
    s2.set_params(**PRM)
    s2.set_flux(nsk.NSK_FLUX_HLLC)
    s2.set_state(U)
    R_dg = s2.rhs()
    assert np.abs(R_fv - R_dg).max() <= 1e-13 * scale(o, U, N, E)
    s.close()
    s2.close()


@pytest.mark.parametrize("pattern", ["dg", "mixed", "fv"])
def test_dirichlet_free_stream(gpu, pattern):
    E, N = 9, 3
    s, o = make_pair(E, N, dirichlet=False, subcell=True)
    Ub = (1.2, 0.15, 1.2)
    s.set_dirichlet(Ub, Ub)
    U = np.zeros(o.shape)
    for v in range(3):
        U[v] = Ub[v]
    s.set_state(U)
    s.set_subcell_flags({"dg": np.zeros(E), "fv": np.ones(E), "mixed": np.arange(E) % 2}[pattern])
    assert np.abs(s.rhs()).max() < 1e-9
    s.close()


@pytest.mark.parametrize("N", [2, 3, 4])
def test_switch_parity(gpu, N):
    """Indicator values, switch decisions and converted states of one pass, from DG and from a
    mixed start."""
    E = 24
    s, o = make_pair(E, N, dirichlet=True)
    x = o.coords()
    U = inputs.riemann_1d(x, 2.0, 0.1, 0.51)  # the jump inside element 12
    U[0] += 0.02 * np.sin(7 * x[0])
    U[2] = U[0].copy()
    for start in (np.zeros(E, np.int32), (np.arange(E) % 5 == 0).astype(np.int32)):
        s.set_state(U)
        s.set_subcell_flags(start)
        s.subcell_switch()
        Ug = s.get_state()
        fg, ig = s.subcell()
        Uo, fo, io = o.fv_switch(U, start)
        assert np.array_equal(fg, fo)
        # far below the thresholds the top mode is a cancellation residue: compare above -11
        big = io > -11
        assert np.all(ig[~big] < -10.5)
        assert np.abs(ig[big] - io[big]).max() < 1e-9
        assert np.abs(Ug - Uo).max() <= 1e-13 * np.abs(Uo).max()
        assert fo[12] == 1
    s.close()


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_riemann_problem_100_steps(gpu, N):
    """The sharp-interface Riemann problem (Sec. 4) on 40 elements: 100 LSRK4 steps with the
    switches before every step (one cooperative launch for the call, its element phases in lane
    groups of 4 lanes up to N = 3 and 8 above), same dt on both sides; flags equal, state within
    1e-10."""
    E = 40
    s, o = make_pair(E, N, dirichlet=True)
    U = inputs.riemann_1d(o.coords(), 2.0, 0.1, 0.5)
    dt = o.timestep(U, 0.1)
    s.set_state(U)
    s.step(dt, 100)
    Ug = s.get_state()
    fg, _ = s.subcell()
    Uo, fo = o.fv_step(U, np.zeros(E, np.int32), dt, 100)
    assert fo.sum() >= 1
    assert np.array_equal(fg, fo)
    for v in range(3):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-10 * np.abs(Uo[v]).max() + 1e-12, v
    s.close()


def test_subcell_api_errors(gpu):
    s = nsk.Solver(2, (4, 4), 3, [0.0, 0.0], [1.0, 1.0], 0, nsk.NSK_FP64)
    s.set_params(**PRM)
    with pytest.raises(RuntimeError):
        s.set_subcell(True)
    with pytest.raises(RuntimeError):
        s.set_dirichlet(LEFT, RIGHT)
    s.close()
    s = nsk.Solver(1, (8,), 3, [0.0], [1.0], 0, nsk.NSK_FP32_MIXED)
    s.set_params(**PRM)
    with pytest.raises(RuntimeError):
        s.set_subcell(True)
    s.close()
    s, o = make_pair(8, 3, dirichlet=True)
    s.set_state(inputs.riemann_1d(o.coords(), 2.0, 0.1, 0.51))
    with pytest.raises(RuntimeError):
        s.lift()
    with pytest.raises(RuntimeError):
        s.set_model(nsk.NSK_MODEL_NSK)
    with pytest.raises(RuntimeError):
        s.set_subcell(True, -8.0, -6.0)  # lower above upper
    s.subcell_switch()
    assert s.subcell()[0].sum() == 1
    with pytest.raises(RuntimeError):
        s.set_subcell(False)  # an element holds sub-cell means
    s.close()


def test_riemann_problem_per_kernel_launches(gpu):
    """4100 elements (above the 4096 of the single cooperative launch): one launch per kernel and
    stage; 30 steps against the oracle."""
    E, N = 4100, 3
    s, o = make_pair(E, N, dirichlet=True)
    U = inputs.riemann_1d(o.coords(), 2.0, 0.1, 0.5)
    dt = o.timestep(U, 0.1)
    s.set_state(U)
    s.step(dt, 30)
    Ug = s.get_state()
    fg, _ = s.subcell()
    Uo, fo = o.fv_step(U, np.zeros(E, np.int32), dt, 30)
    assert fo.sum() >= 1 and np.array_equal(fg, fo)
    for v in range(3):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-10 * np.abs(Uo[v]).max() + 1e-12, v
    s.close()


def test_riemann_problem_adaptive_dt(gpu):
    """dt <= 0 (CFL recomputed before every step, per-kernel launches) against the oracle taking
    its own time step before each of its steps."""
    E, N = 40, 2
    s, o = make_pair(E, N, dirichlet=True)
    U = inputs.riemann_1d(o.coords(), 2.0, 0.1, 0.5)
    s.set_state(U)
    s.step(-0.1, 30)
    Ug = s.get_state()
    fg, _ = s.subcell()
    Uo, fo = U, np.zeros(E, np.int32)
    for _ in range(30):
        Uo, fo = o.fv_step(Uo, fo, o.timestep(Uo, 0.1), 1)
    assert np.array_equal(fg, fo)
    for v in range(3):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-10 * np.abs(Uo[v]).max() + 1e-12, v
    s.close()


def test_riemann_problem_large_mesh_unsplit_launches(gpu):
    """70,000 elements: per-kernel launches without the DG/FV split of small meshes (above
    65,536 elements); 5 steps against the oracle."""
    E, N = 70000, 3
    s, o = make_pair(E, N, dirichlet=True)
    U = inputs.riemann_1d(o.coords(), 2.0, 0.1, 0.5)
    dt = o.timestep(U, 0.1)
    s.set_state(U)
    s.step(dt, 5)
    Ug = s.get_state()
    fg, _ = s.subcell()
    Uo, fo = o.fv_step(U, np.zeros(E, np.int32), dt, 5)
    assert fo.sum() >= 1 and np.array_equal(fg, fo)
    for v in range(3):
        assert np.abs(Ug[v] - Uo[v]).max() <= 1e-10 * np.abs(Uo[v]).max() + 1e-12, v
    s.close()
