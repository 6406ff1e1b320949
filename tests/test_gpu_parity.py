"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64 path): the two sides evaluate the same formulas in a
different order and with fused multiply-adds on the GPU, so single operators
agree to a few hundred ulps of the largest term they combine; we require
1e-12 relative to the scale of each output. After 100 LSRK4 steps the
relative L-infinity error of every variable against its own scale
(max |U_gpu[v] - U_orc[v]| / max |U_orc[v]|, tolerances.state_rel_err) must be
<= 1e-11.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs, nsk
from tolerances import rhs_tolerance, state_rel_err

pytestmark = pytest.mark.gpu


def make_pair(dim, ne, N, nt=0, lo=None, hi=None, precision=nsk.NSK_FP64, **params):
    prm = dict(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3)
    cdiss = params.pop("c_dissipation", 0)
    flux = params.pop("flux", nsk.NSK_FLUX_LF)
    prm.update(params)
    lo = lo or [0.0] * dim
    hi = hi or [1.0] * dim
    s = nsk.Solver(dim, ne, N, lo, hi, nt, precision)
    s.set_params(**prm)
    if cdiss:
        s.set_c_dissipation(True)
    if flux != nsk.NSK_FLUX_LF:
        s.set_flux(flux)
    o = O.Oracle(dim, ne, lo, hi, N, nt, c_dissipation=cdiss, flux=flux, **prm)
    return s, o


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


OPERATOR_CASES = [
    # dim, nelem, N, node type: several blocks per launch with a ragged tail
    (1, (100,), 3, 0), (1, (13,), 4, 1), (1, (7,), 1, 0), (1, (9,), 5, 0),
    (2, (7, 5), 4, 0), (2, (12, 9), 2, 1), (2, (5, 6), 3, 0),
    (3, (5, 3, 3), 3, 0), (3, (4, 3, 5), 2, 1), (3, (3, 3, 2), 4, 0), (3, (2, 3, 2), 5, 0),
]


@pytest.mark.parametrize("dim,ne,N,nt", OPERATOR_CASES)
def test_node_coords_match(gpu, dim, ne, N, nt):
    s, o = make_pair(dim, ne, N, nt, hi=[1.0, 0.8, 1.3][:dim])
    assert np.abs(s.node_coords() - o.coords()).max() < 1e-14
    s.close()


@pytest.mark.parametrize("dim,ne,N,nt", OPERATOR_CASES)
def test_lift_parity(gpu, dim, ne, N, nt):
    s, o = make_pair(dim, ne, N, nt, hi=[1.0, 0.8, 1.3][:dim])
    U = inputs.random_state(o.shape, seed=100 + dim * 10 + N)
    s.set_state(U)
    Qg, Qo = s.lift(), o.lift(U)
    for c in range(o.nq):
        scale = np.abs(Qo[c]).max() + 1e-3 * np.abs(Qo).max()
        assert np.abs(Qg[c] - Qo[c]).max() <= 1e-12 * scale, c
    s.close()


@pytest.mark.parametrize("dim,ne,N,nt", OPERATOR_CASES)
def test_rhs_parity(gpu, dim, ne, N, nt):
    s, o = make_pair(dim, ne, N, nt, hi=[1.0, 0.8, 1.3][:dim], mu=2e-2, kappa=1e-3)
    U = inputs.random_state(o.shape, seed=200 + dim * 10 + N)
    s.set_state(U)
    Rg, Ro = s.rhs(), o.rhs(U)
    tol = rhs_tolerance(o, U, Ro)
    for v in range(o.nvar):
        err = np.abs(Rg[v] - Ro[v]).max()
        assert err <= tol[v], (v, err, tol[v])
    s.close()


def test_rhs_parity_c_dissipation(gpu):
    s, o = make_pair(2, (6, 5), 3, 0, c_dissipation=1)
    U = inputs.random_state(o.shape, seed=7)
    s.set_state(U)
    assert rel_err(s.rhs(), o.rhs(U)) < 1e-12
    s.close()


HLLC_CASES = [(1, (13,), 4, 1), (2, (7, 5), 4, 0), (2, (5, 6), 3, 0), (3, (5, 3, 3), 3, 0), (3, (3, 3, 2), 4, 0)]


@pytest.mark.parametrize("dim,ne,N,nt", HLLC_CASES)
@pytest.mark.parametrize("regime", ["subsonic", "transonic"])
def test_rhs_parity_hllc(gpu, dim, ne, N, nt, regime):
    """HLLC face flux. Subsonic: alpha = 1e3 (sound speed ~ 35, |v| < 0.3: every face in the star
    region, contacts moving either way). Transonic: alpha = 2 (sound speed 1.0..1.6) and |v| up
    to 3, so faces take all four branches of the solver (F_L, L*, R*, F_R)."""
    prm = dict(mu=2e-2, kappa=1e-3) if regime == "subsonic" else dict(mu=2e-2, kappa=1e-3, alpha=2.0, beta=1.0)
    s, o = make_pair(dim, ne, N, nt, hi=[1.0, 0.8, 1.3][:dim], flux=nsk.NSK_FLUX_HLLC, **prm)
    U = inputs.random_state(o.shape, seed=300 + dim * 10 + N)
    if regime == "transonic":
        U[1:dim + 1] *= 15.0
    s.set_state(U)
    Rg, Ro = s.rhs(), o.rhs(U)
    tol = rhs_tolerance(o, U, Ro)
    for v in range(o.nvar):
        err = np.abs(Rg[v] - Ro[v]).max()
        assert err <= tol[v], (v, err, tol[v])
    s.close()


@pytest.mark.parametrize("name", ["droplets2d", "collision3d"])
def test_step_parity_100_hllc(gpu, name):
    """100 LSRK4 steps with the HLLC flux: rel. L-inf error <= 1e-11."""
    s, o, U = _physical_case(name, flux=nsk.NSK_FLUX_HLLC)
    dt = o.timestep(U, 0.5)
    s.set_state(U)
    s.step(dt, 100)
    Ug = s.get_state()
    Uo = o.step(U, dt, 100)
    err, per_var = state_rel_err(Ug, Uo)
    assert err <= 1e-11, per_var
    s.close()


def test_free_stream_gpu(gpu):
    s, o = make_pair(3, (4, 3, 5), 3, 0, hi=[1.0, 0.7, 1.3])
    U = np.zeros(o.shape)
    U[0], U[1], U[2], U[3], U[4] = 1.3, 0.52, 0.13, -0.26, 1.3
    s.set_state(U)
    assert np.abs(s.rhs()).max() < 1e-8
    s.close()


def _physical_case(name, flux=nsk.NSK_FLUX_LF):
    rv, rl, _ = O.maxwell(0.85)
    if name == "slab1d_gll":
        s, o = make_pair(1, (64,), 3, 1, flux=flux)
        U = inputs.slab_1d(o.coords(), rv, rl, 1e-4)
    elif name == "slab1d_gl_paper_params":
        s, o = make_pair(1, (64,), 3, 0, alpha=100.0, beta=1e-2, mu=1e-2, flux=flux)
        U = inputs.slab_1d(o.coords(), rv, rl, 1e-4)
    elif name == "droplets2d":
        s, o = make_pair(2, (16, 16), 4, 0, mu=2e-3, flux=flux)
        U = inputs.droplets(o.coords(), ((0.35, 0.5), (0.65, 0.5)), (0.15, 0.12), rv, rl, 1e-4)
        U = inputs.add_density_noise(U, 1e-4)
    elif name == "collision3d":
        s, o = make_pair(3, (7, 6, 5), 3, 0, flux=flux)
        v = inputs.collision_velocity(40.0, 0.2, 1e-4, rv, rl)
        U = inputs.head_on_collision(o.coords(), v, 0.2, rho_vap=rv, rho_liq=rl, kappa=1e-4)
    else:
        raise KeyError(name)
    return s, o, U


@pytest.mark.parametrize("name", ["slab1d_gll", "slab1d_gl_paper_params", "droplets2d", "collision3d"])
def test_step_parity_100(gpu, name):
    """100 LSRK4 steps at the oracle's CFL-0.5 step: rel. L-inf error <= 1e-11."""
    s, o, U = _physical_case(name)
    dt = o.timestep(U, 0.5)
    s.set_state(U)
    assert abs(s.compute_dt(0.5) - dt) <= 1e-13 * dt
    s.step(dt, 100)
    Ug = s.get_state()
    Uo = o.step(U, dt, 100)
    err, per_var = state_rel_err(Ug, Uo)
    assert err <= 1e-11, per_var
    # conservation and diagnostics agree too
    mg, eg, lg = s.diagnostics()
    mo, eo, lo_ = o.diagnostics(Uo)
    assert abs(mg - mo) <= 1e-12 * abs(mo)
    assert abs(eg - eo) <= 1e-10 * abs(eo)
    assert abs(lg - lo_) <= 1e-6 * lo_ + 1e-14
    s.close()


def test_adaptive_dt_step_matches_fixed(gpu):
    s, o, U = _physical_case("droplets2d")
    s.set_state(U)
    s.step(-0.5, 3)
    Ua = s.get_state()
    Uo = U
    for _ in range(3):
        Uo = o.step(Uo, o.timestep(Uo, 0.5), 1)
    assert rel_err(Ua, Uo) < 1e-12
    s.close()


def test_device_pointer_path(gpu):
    import torch

    s, o = make_pair(2, (5, 4), 3, 0)
    U = inputs.random_state(o.shape, seed=3)
    Ut = torch.from_numpy(U).to(gpu)
    s.set_state(Ut)
    R_dev = torch.empty_like(Ut)
    s.rhs(out=R_dev)
    torch.cuda.synchronize()
    R_host = s.rhs()
    assert np.array_equal(R_dev.cpu().numpy(), R_host)
    back = torch.empty_like(Ut)
    s.get_state(out=back)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), U)
    s.close()


def test_nonphysical_state_is_reported(gpu):
    s, o = make_pair(2, (4, 4), 3, 0)
    U = inputs.random_state(o.shape, seed=4)
    U[0, 5, 3] = 3.5  # beyond the co-volume limit 1/b = 3 of the VdW fluid
    s.set_state(U)
    with pytest.raises(nsk.NskError) as ei:
        s.rhs()
    assert ei.value.code == nsk.NSK_ERR_NONPHYSICAL
    # the context stays usable once a valid state is set again
    U[0, 5, 3] = 1.2
    s.set_state(U)
    s.rhs()
    s.close()


def test_call_order_and_parameter_checks(gpu):
    s = nsk.Solver(2, (3, 3), 2)
    with pytest.raises(nsk.NskError) as ei:
        s.rhs()
    assert ei.value.code == nsk.NSK_ERR_STATE
    with pytest.raises(nsk.NskError) as ei:
        s.set_params(T=0.85, kappa=1e-4, alpha=0.45, beta=1e-3, mu=1e-3)  # alpha <= alpha_* = 0.45
    assert ei.value.code == nsk.NSK_ERR_ARG
    s.set_params(T=0.85, kappa=1e-4, alpha=0.46, beta=1e-3, mu=1e-3)
    s.close()


def test_launch_counter_and_profile(gpu):
    s, o, U = _physical_case("collision3d")
    s.set_state(U)
    n0 = s.launch_count
    s.set_profiling(True)
    s.step(1e-7, 2)
    prof = s.get_profile(reset=True)
    # one prolongation pass per call: later stages take the traces the volume kernel wrote
    assert prof["k_prolong"][1] == 1
    assert prof["k_lift"][1] == 10 and prof["k_face"][1] == 10 and prof["k_volume"][1] == 10
    assert s.launch_count - n0 == 1 + 2 * 5 * 3
    assert all(ms > 0 for ms, _ in prof.values())
    s.set_schedule(128, True)
    n0 = s.launch_count
    s.step(1e-7, 1)
    prof = s.get_profile(reset=True)
    assert prof["k_face"][1] == 0 and prof["k_volume"][1] == 5 and prof["k_prolong"][1] == 1
    assert s.launch_count - n0 == 1 + 5 * 2
    s.set_schedule(256, 2)  # lean stage: the viscous-trace lifting and the volume kernel
    n0 = s.launch_count
    s.step(1e-7, 1)
    prof = s.get_profile(reset=True)
    assert prof["k_face"][1] == 0 and prof["k_lift"][1] == 5 and prof["k_volume"][1] == 5
    assert s.launch_count - n0 == 1 + 5 * 2
    s.close()


@pytest.mark.parametrize("name", ["droplets2d", "collision3d"])
@pytest.mark.parametrize("precision", [nsk.NSK_FP64, nsk.NSK_FP32_MIXED])
def test_lean_schedule_residual_and_steps(gpu, name, precision):
    """The lean two-launch stage (lifting recomputed by the volume kernel) against the oracle:
    residual per variable within the residual tolerance (FP32: the FP32 operator's bound on the
    FP32-rounded state), and in FP64 100 steps within 1e-11 of each variable's scale."""
    s, o, U = _physical_case(name)
    if precision == nsk.NSK_FP32_MIXED:
        s.close()
        s = nsk.Solver(o.dim, o.nelem, o.N, [0.0] * o.dim, [1.0] * o.dim, 0, precision)
        s.set_params(T=0.85, kappa=o.s.kappa, alpha=o.s.alpha, beta=o.s.beta, mu=o.s.mu)
    s.set_schedule(256, 2)
    s.set_state(U)
    Ul = U if precision == nsk.NSK_FP64 else U.astype(np.float32).astype(np.float64)  # as the context stores it
    Rg, Ro = s.rhs(), o.rhs(Ul)
    tol = rhs_tolerance(o, Ul, Ro)
    for v in range(o.nvar):
        bound = tol[v] if precision == nsk.NSK_FP64 else \
            tol[v] * (2.0**-24 / 2.0**-53) * 0.5 + 1e-5 * np.abs(Ro[v]).max()  # the FP32 operator's bound
        err = float(np.abs(Rg[v] - Ro[v]).max())
        assert err <= bound, (v, err, bound)
    if precision == nsk.NSK_FP64:
        dt = o.timestep(U, 0.5)
        s.set_state(U)
        s.step(dt, 100)
        err, per_var = state_rel_err(s.get_state(), o.step(U, dt, 100))
        assert err <= 1e-11, per_var
    s.close()


# ---------------------------------------------------------------- full size

def _tile(Usmall, small_ne, reps):
    """State of a periodic box made of reps[k] copies of a small periodic box (same element size)."""
    nvar, Es, npe = Usmall.shape
    nx, ny, nz = small_ne
    big_ne = (nx * reps[0], ny * reps[1], nz * reps[2])
    A = Usmall.reshape(nvar, nz, ny, nx, npe)
    B = np.tile(A, (1, reps[2], reps[1], reps[0], 1))
    return np.ascontiguousarray(B.reshape(nvar, -1, npe)), big_ne


def test_full_size_head_on_collision_tiled(gpu):
    """At the 64^3-element, N=3 size the benchmark times (16.8M nodes x 5 variables), a state
    that repeats a 4^3-element periodic box 16 times per direction must give, in every element,
    the residual and the 3-step solution the oracle computes on the small box."""
    small = (4, 4, 4)
    reps = (16, 16, 16)
    h = 1.0 / 64
    o = O.Oracle(3, small, (0, 0, 0), (4 * h,) * 3, 3, 0)
    x = o.coords() * 16.0  # any smooth periodic pattern on the small box
    rv, rl, _ = O.maxwell(0.85)
    U = inputs.droplets(x, ((0.5, 0.5, 0.5),), (0.25,), rv, rl, 1e-4 * 256)
    U[1] = U[0] * 0.1 * np.sin(2 * np.pi * x[1])
    U[2] = U[0] * 0.05 * np.cos(2 * np.pi * x[2])
    U[3] = -U[0] * 0.07 * np.sin(2 * np.pi * x[0])
    U[4] = U[0] * (1 + 1e-3 * np.cos(2 * np.pi * (x[0] + x[1])))
    Ubig, big_ne = _tile(U, small, reps)
    s = nsk.Solver(3, big_ne, 3, [0, 0, 0], [1, 1, 1], 0)
    s.set_params(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3)
    s.set_state(Ubig)
    Rg = s.rhs()
    Rs = o.rhs(U)
    tol = rhs_tolerance(o, U, Rs)
    Ro, _ = _tile(Rs, small, reps)
    for v in range(5):
        err = float(np.abs(Rg[v] - Ro[v]).max())
        assert err <= tol[v], (v, err, tol[v])
    dt = o.timestep(U, 0.5)
    s.step(dt, 3)
    Ug = s.get_state()
    Uo, _ = _tile(o.step(U, dt, 3), small, reps)
    err, per_var = state_rel_err(Ug, Uo)
    assert err <= 1e-12, per_var
    s.close()


@pytest.mark.parametrize("name", ["slab1d_gll", "slab1d_gl_paper_params"])
def test_single_block_schedule(gpu, name):
    """The single-block schedule (a small mesh's whole nsk_step call in one launch, arrays in shared
    memory): one launch per call, 100 steps within 1e-11 of the oracle per variable, and the same
    bits as the separate face pass (residual and steps; the residual's oracle parity is the
    separate pass's)."""
    s, o, U = _physical_case(name)
    dt = o.timestep(U, 0.5)
    s.set_schedule(256, 3)
    s.set_state(U)
    s.set_profiling(True)
    n0 = s.launch_count
    s.step(dt, 100)
    prof = s.get_profile(reset=True)
    assert s.launch_count - n0 == 1 and prof["k_block"][1] == 1
    Ub = s.get_state()
    err, per_var = state_rel_err(Ub, o.step(U, dt, 100))
    assert err <= 1e-11, per_var
    s.set_state(U)
    Rg = s.rhs()
    s.set_schedule(256, 0)
    s.set_state(U)
    assert np.array_equal(s.rhs(), Rg)
    s.step(dt, 100)
    assert np.array_equal(s.get_state(), Ub)
    s.set_profiling(False)
    s.close()
