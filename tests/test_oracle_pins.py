"""Pins of the CPU oracle to what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, library routines, textbook order conditions,
exactness and conservation properties, brute-force symmetry. A plausible slip
in the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import math
from pathlib import Path

import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs

GOLDEN = Path(__file__).resolve().parent / "golden"


def _golden_rows(name):
    rows = []
    for line in (GOLDEN / name).read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------- thermodynamics

def test_maxwell_densities_match_paper():
    """Sec. 4.1.1 prints rho_vap = 0.3197, rho_liq = 1.8071 at T = 0.85."""
    (T, rv_p, rl_p), = [tuple(map(float, r)) for r in _golden_rows("maxwell_T085.txt")]
    rv, rl, ps = O.maxwell(T)
    assert abs(rv - rv_p) < 5e-5 and abs(rl - rl_p) < 5e-5
    # equal pressure and equal chemical potential (Maxwell construction, Sec. 2.1)
    assert abs(O.pressure(T, rv) - O.pressure(T, rl)) < 1e-13
    assert abs(O.chem_potential(T, rv) - O.chem_potential(T, rl)) < 1e-12
    # equal-area rule: integral of p dV from v_l to v_v equals p_sat (v_v - v_l), V = 1/rho
    Vs = np.linspace(1 / rl, 1 / rv, 200001)
    integral = np.trapezoid([O.pressure(T, 1 / V) for V in Vs], Vs)
    assert abs(integral - ps * (1 / rv - 1 / rl)) < 1e-8


def test_pressure_closed_form_and_derivatives():
    """Eq. (vdw_p) with a=3, b=1/3, R=8/3: p = 8 T rho/(3-rho) - 3 rho^2; p = rho W' - W."""
    T = 0.85
    for rho in (0.1, 0.5, 1.0, 1.7, 2.5):
        assert abs(O.pressure(T, rho) - (8 * T * rho / (3 - rho) - 3 * rho**2)) < 1e-13
        h = 1e-5
        dW = (O.free_energy(T, rho + h) - O.free_energy(T, rho - h)) / (2 * h)
        assert abs(rho * dW - O.free_energy(T, rho) - O.pressure(T, rho)) < 1e-8 * max(1.0, abs(dW))
        dp = (O.pressure(T, rho + h) - O.pressure(T, rho - h)) / (2 * h)
        assert abs(dp - O.dpressure(T, rho)) < 1e-8 * max(1.0, abs(dp))


def test_spinodal_and_alpha_star():
    """alpha_* = |min W''|/2 (Eq. alpha_fullyhyperbolic_limit); for the reduced VdW fluid
    W'' = 24T/(rho (3-rho)^2) - 6 is smallest at rho = 1, so alpha_* = 3 (1 - T) = 0.45."""
    sv, sl, astar = O.spinodal(0.85)
    assert abs(astar - 0.45) < 1e-12
    assert abs(O.dpressure(0.85, sv)) < 1e-12 and abs(O.dpressure(0.85, sl)) < 1e-12
    rv, rl, _ = O.maxwell(0.85)
    assert rv < sv < 1.0 < sl < rl
    # mean density contour of Sec. 4.2 (printed 1.0634) is the mean of the Maxwell states
    assert abs(0.5 * (rv + rl) - 1.0634) < 5e-5


def test_young_laplace_reproduces_hoc_table():
    """All eight phase densities of the HOC table (Sec. 4.3) follow from Eq. (hoc_initialpressures)
    with r = 0.1, rho_c = 1 and sigma = 2 r rho_c v_rel^2 / We_coll."""
    for case, Re, We, eps, gam, v, rl_p, rv_p in _golden_rows("hoc_table.txt"):
        sigma = 2 * 0.1 * 1.0 * float(v) ** 2 / float(We)
        rl, rv = O.young_laplace(0.85, sigma, 0.1)
        assert abs(rl - float(rl_p)) < 6e-5, case
        assert abs(rv - float(rv_p)) < 6e-5, case
        # the table's gamma is 1 / (We eps^2) with We = 6000 for HOC2/2A/3
        if case != "HOC1":
            assert abs(float(gam) - 1.0 / (6000 * float(eps) ** 2)) / float(gam) < 1e-3


# ---------------------------------------------------------------- basis

@pytest.mark.parametrize("N", range(1, 8))
def test_gauss_legendre_nodes_match_numpy(N):
    xi, w = O.nodes(N, O.NODES_GAUSS)
    xr, wr = np.polynomial.legendre.leggauss(N + 1)
    assert np.allclose(xi, xr, atol=1e-15, rtol=0) and np.allclose(w, wr, atol=1e-15, rtol=0)


def test_gauss_lobatto_closed_forms():
    xi, w = O.nodes(2, O.NODES_LOBATTO)
    assert np.allclose(xi, [-1, 0, 1], atol=1e-16) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    xi, w = O.nodes(3, O.NODES_LOBATTO)
    s = 1 / math.sqrt(5)
    assert np.allclose(xi, [-1, -s, s, 1], atol=1e-15) and np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    xi, w = O.nodes(4, O.NODES_LOBATTO)
    s = math.sqrt(3 / 7)
    assert np.allclose(xi, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("node_type", [O.NODES_GAUSS, O.NODES_LOBATTO])
@pytest.mark.parametrize("N", range(1, 7))
def test_quadrature_and_derivative_exactness(N, node_type):
    xi, w = O.nodes(N, node_type)
    D, Lm, Lp = O.lagrange_tables(N, xi)
    exact_deg = 2 * N + 1 if node_type == O.NODES_GAUSS else 2 * N - 1
    for m in range(exact_deg + 1):  # quadrature exact up to its degree
        assert abs(np.dot(w, xi**m) - (2 / (m + 1) if m % 2 == 0 else 0)) < 1e-14
    for m in range(N + 1):  # D exact on monomials of degree <= N; interpolation to +-1 exact
        d_exact = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        assert np.allclose(D @ xi**m, d_exact, atol=1e-12, rtol=0)
        assert abs(Lp @ xi**m - 1.0) < 1e-13 and abs(Lm @ xi**m - (-1.0) ** m) < 1e-13


# ---------------------------------------------------------------- time integration

def _butcher_from_2n(A, B):
    """Butcher tableau of the 2N-storage scheme K_i = A_i K_{i-1} + dt f(Y_i), U_i = U_{i-1} + B_i K_i."""
    s = len(A)
    a = np.zeros((s + 1, s))
    for i in range(1, s + 1):          # row i: Y_{i+1} = U_i
        for j in range(i):
            acc = 0.0
            for l in range(j, i):
                prod = 1.0
                for m in range(j + 1, l + 1):
                    prod *= A[m]
                acc += B[l] * prod
            a[i, j] = acc
    return a[:s], a[s]


def test_lsrk4_order_conditions():
    """The eight fourth-order conditions hold for the Carpenter-Kennedy 2N coefficients,
    and the abscissae C equal the row sums of the equivalent Butcher tableau."""
    A, B, Cc = O.lsrk4_coeffs()
    a, b = _butcher_from_2n(A, B)
    c = a.sum(axis=1)
    assert np.allclose(c, Cc, atol=1e-15)
    conds = [
        (b.sum(), 1.0), (b @ c, 1 / 2), (b @ c**2, 1 / 3), (b @ (a @ c), 1 / 6),
        (b @ c**3, 1 / 4), (b @ (c * (a @ c)), 1 / 8), (b @ (a @ c**2), 1 / 12), (b @ (a @ (a @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-14


def test_lsrk4_relaxation_closed_form_and_order():
    """A spatially uniform state with c != rho reduces model II to c' = (alpha/beta)(rho - c)
    (rho, m stay constant): c(t) = rho + (c0 - rho) exp(-alpha t / beta). The oracle's residual
    and time stepper reproduce it with fourth-order temporal convergence."""
    # large elements keep the explicit step far inside the convective and viscous limits
    orc = O.Oracle(2, (3, 2), (0, 0), (60.0, 40.0), 2, alpha=2.0, beta=1.0, kappa=1e-3, mu=1e-3)
    U0 = np.zeros(orc.shape)
    U0[0], U0[1], U0[2], U0[3] = 1.2, 0.3, -0.1, 1.5
    R = orc.rhs(U0)
    assert np.allclose(R[:3], 0, atol=1e-12) and np.allclose(R[3], 2.0 * (1.2 - 1.5), atol=1e-12)
    tend, errs = 1.0, []
    for nsteps in (8, 16, 32):
        U = orc.step(U0, tend / nsteps, nsteps)
        exact = 1.2 + 0.3 * math.exp(-2.0 * tend)
        errs.append(abs(U[3, 0, 0] - exact))
        assert np.allclose(U[0], 1.2, atol=1e-13) and np.allclose(U[1], 0.3, atol=1e-13)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.8 < o < 4.3 for o in orders), (errs, orders)


# ---------------------------------------------------------------- residual properties

def _cases():
    return [
        (1, (6,), 3, O.NODES_GAUSS), (1, (5,), 4, O.NODES_LOBATTO),
        (2, (4, 3), 3, O.NODES_GAUSS), (2, (3, 4), 2, O.NODES_LOBATTO),
        (3, (3, 2, 2), 2, O.NODES_GAUSS), (3, (2, 3, 2), 3, O.NODES_LOBATTO),
    ]


@pytest.mark.parametrize("dim,ne,N,nt", _cases())
def test_free_stream_preservation(dim, ne, N, nt):
    """A constant state with c = rho is a steady solution: R = 0 to round-off, also on
    anisotropic (non-cubic) elements."""
    orc = O.Oracle(dim, ne, [0.0] * dim, [1.0, 0.7, 1.3][:dim], N, nt)
    U = np.zeros(orc.shape)
    U[0] = 1.3
    for a in range(dim):
        U[1 + a] = 1.3 * (0.4 - 0.3 * a)
    U[-1] = 1.3
    R = orc.rhs(U)
    scale = 1e3  # magnitude of p_alpha at rho = 1.3, alpha = 1e3
    assert np.abs(R).max() < 1e-13 * scale * max(ne) * (N + 1) ** 2


def _global_poly(x, coeffs):
    """Tensor-product polynomial sum_c prod_k x_k^{p_k} with coefficients from coeffs."""
    out = np.zeros(x.shape[1:])
    for c, pw in coeffs:
        t = np.full(x.shape[1:], c)
        for k, p in enumerate(pw):
            t = t * x[k] ** p
        out += t
    return out


def _grad_poly(x, coeffs, k):
    out = np.zeros(x.shape[1:])
    for c, pw in coeffs:
        if pw[k] == 0:
            continue
        t = np.full(x.shape[1:], c * pw[k])
        for q, p in enumerate(pw):
            t = t * x[q] ** (p - 1 if q == k else p)
        out += t
    return out


@pytest.mark.parametrize("dim,ne,N,nt", [
    (1, (6,), 3, O.NODES_GAUSS), (1, (5,), 4, O.NODES_LOBATTO),
    (2, (4, 3), 3, O.NODES_GAUSS), (2, (3, 4), 2, O.NODES_LOBATTO),
    (3, (3, 4, 3), 2, O.NODES_GAUSS), (3, (3, 3, 3), 3, O.NODES_LOBATTO),
])
def test_lifting_exact_for_polynomials(dim, ne, N, nt):
    """BR1 with the central flux returns the exact gradient of a field that is one global
    polynomial of degree <= N per direction: in every element away from the periodic seam,
    the traces of both sides agree, so w* equals the element's own trace (Sec. 3.1)."""
    orc = O.Oracle(dim, ne, [0.0] * dim, [1.0] * dim, N, nt)
    x = orc.coords()
    rng = np.random.default_rng(3)
    polys = []
    for q in range(dim + 1):
        terms = []
        for _ in range(4):
            pw = tuple(int(rng.integers(0, N + 1)) for _ in range(dim))
            terms.append((float(rng.uniform(-0.5, 0.5)), pw))
        polys.append(terms)
    rho0 = 1.1
    U = np.zeros(orc.shape)
    U[0] = rho0
    for a in range(dim):
        U[1 + a] = rho0 * _global_poly(x, polys[a])
    U[-1] = 1.0 + _global_poly(x, polys[dim])
    Q = orc.lift(U)
    # interior elements: no face on the periodic seam
    interior = np.ones(orc.E, bool)
    for e in range(orc.E):
        r = e
        for k in range(dim):
            ck = r % ne[k]
            r //= ne[k]
            if ck == 0 or ck == ne[k] - 1:
                interior[e] = False
    assert interior.any()
    for k in range(dim):
        for w in range(dim + 1):
            exact = _grad_poly(x, polys[w], k)
            got = Q[k * (dim + 1) + w]
            assert np.allclose(got[interior], exact[interior], atol=1e-11, rtol=0), (k, w)


def test_lifting_c_exact_with_varying_density():
    """c is lifted directly, so its gradient is exact whatever rho does."""
    orc = O.Oracle(2, (4, 4), (0, 0), (1, 1), 3)
    x = orc.coords()
    U = inputs.random_state(orc.shape, seed=5)
    U[-1] = 1.0 + 0.3 * x[0] ** 3 - 0.2 * x[0] * x[1] ** 2
    Q = orc.lift(U)
    inner = [5, 6, 9, 10]
    assert np.allclose(Q[0 * 3 + 2][inner], (0.9 * x[0] ** 2 - 0.2 * x[1] ** 2)[inner], atol=1e-11)
    assert np.allclose(Q[1 * 3 + 2][inner], (-0.4 * x[0] * x[1])[inner], atol=1e-11)


def _quad_weights(orc):
    h = [(orc.hi[k] - orc.lo[k]) / orc.nelem[k] for k in range(orc.dim)]
    wq = np.ones(orc.npe)
    for n in range(orc.npe):
        r = n
        for k in range(orc.dim):
            wq[n] *= orc.w[r % orc.np] * h[k] / 2
            r //= orc.np
    return wq


@pytest.mark.parametrize("dim,ne,N,nt", _cases())
def test_mass_conservation(dim, ne, N, nt):
    """No mass source and a single-valued face flux on periodic faces: sum w J d(rho)/dt = 0,
    and the mass of the LSRK solution is constant."""
    orc = O.Oracle(dim, ne, [0.0] * dim, [1.0] * dim, N, nt, alpha=50.0, beta=0.05, kappa=1e-3, mu=1e-2)
    U = inputs.random_state(orc.shape, seed=11)
    R = orc.rhs(U)
    wq = _quad_weights(orc)
    flux_scale = np.abs(R[0]).max()
    assert abs((R[0] * wq).sum()) < 1e-13 * flux_scale
    m0 = orc.diagnostics(U)[0]
    U2 = orc.step(U, 1e-5, 3)
    assert abs(orc.diagnostics(U2)[0] - m0) < 1e-14 * abs(m0) * 10


def test_momentum_source_balances_pressure_at_equilibrium_limit():
    """Model II momentum source alpha rho grad c cancels the alpha rho^2/2 part of p_alpha
    when c = rho (Eq. modified_pressure): with alpha large and c = rho the residual equals
    that of alpha = 0 up to the O(1) discretisation of alpha rho (grad c - grad rho)."""
    kw = dict(dim=1, nelem=(16,), lo=(0,), hi=(1,), N=4)
    o1 = O.Oracle(**kw, alpha=1e3)
    o2 = O.Oracle(**kw, alpha=2e3)
    x = o1.coords()
    U = np.zeros(o1.shape)
    U[0] = 1.4 + 0.1 * np.sin(2 * np.pi * x[0])
    U[-1] = U[0]
    R1, R2 = o1.rhs(U), o2.rhs(U)
    # alpha enters the momentum residual only through alpha * (discrete rho grad c - d/dx rho^2/2),
    # which is a consistent discretisation of zero: doubling alpha changes R by far less than alpha.
    assert np.abs(R2[1] - R1[1]).max() < 1e-3 * 1e3
    assert np.abs(R1[1]).max() < 1.0


def test_dimension_consistency_3d_equals_1d():
    """A 3D state constant in y and z gives the 1D residual in every y-z column (brute force)."""
    o1 = O.Oracle(1, (5,), (0,), (1,), 3, kappa=1e-3, mu=2e-3)
    o3 = O.Oracle(3, (5, 2, 3), (0, 0, 0), (1, 0.5, 2.0), 3, kappa=1e-3, mu=2e-3)
    U1 = inputs.random_state(o1.shape, seed=2)
    U3 = np.zeros(o3.shape)
    np1 = o1.np
    for e in range(o3.E):
        ex = e % 5
        for n in range(o3.npe):
            i = n % np1
            U3[0, e, n] = U1[0, ex, i]
            U3[1, e, n] = U1[1, ex, i]
            U3[4, e, n] = U1[2, ex, i]
    R1, R3 = o1.rhs(U1), o3.rhs(U3)
    for e in range(o3.E):
        ex = e % 5
        for n in range(o3.npe):
            i = n % np1
            assert abs(R3[0, e, n] - R1[0, ex, i]) < 1e-9
            assert abs(R3[1, e, n] - R1[1, ex, i]) < 1e-9
            assert abs(R3[4, e, n] - R1[2, ex, i]) < 1e-9
            assert abs(R3[2, e, n]) < 1e-9 and abs(R3[3, e, n]) < 1e-9


def test_transpose_symmetry_2d():
    """Swapping x <-> y (and the two momentum components) maps the residual the same way."""
    ne = (3, 3)
    o = O.Oracle(2, ne, (0, 0), (1, 1), 3, kappa=1e-3, mu=3e-2)
    U = inputs.random_state(o.shape, seed=9)
    npn = o.np

    def transpose(A, swap):
        B = np.empty_like(A)
        for e in range(o.E):
            ex, ey = e % 3, e // 3
            et = ey + 3 * ex
            for n in range(o.npe):
                i, j = n % npn, n // npn
                nt = j + npn * i
                B[:, et, nt] = A[:, e, n]
        if swap:
            B[[1, 2]] = B[[2, 1]]
        return B

    R = o.rhs(U)
    Rt = o.rhs(transpose(U, True))
    assert np.allclose(Rt, transpose(R, True), atol=1e-9, rtol=1e-12)


def test_energy_decay_static_interface():
    """Total energy of the relaxation model (Eq. pararelax_elliptical_energy_dynamic) does not
    increase (Sec. 4.1.1, Sec. 4.2): a 1D slab relaxing from its tanh profile."""
    rv, rl, _ = O.maxwell(0.85)
    orc = O.Oracle(1, (24,), (0,), (1,), 3, O.NODES_GAUSS, alpha=100.0, beta=1e-2, kappa=1e-4 * 4, mu=1e-2)
    U = inputs.slab_1d(orc.coords(), rv, rl, kappa=1e-4 * 4)
    dt = orc.timestep(U, 0.5)
    energies = [orc.diagnostics(U)[1]]
    for _ in range(30):
        U = orc.step(U, dt, 5)
        energies.append(orc.diagnostics(U)[1])
    diffs = np.diff(energies)
    assert (diffs <= 1e-12 * abs(energies[0])).all(), diffs
    assert energies[-1] < energies[0]


def test_timestep_bounds():
    """dt is the minimum of the convective, parabolic (Eq. numerics_dfl) and source bounds."""
    orc = O.Oracle(2, (4, 8), (0, 0), (1, 1), 3, alpha=1e3, beta=1e-3, kappa=1e-4, mu=1e-3)
    U = np.zeros(orc.shape)
    U[0], U[1], U[3] = 1.0, 0.5, 1.0
    a = math.sqrt(O.dpressure(0.85, 1.0) + 1e3 * 1.0)
    conv = 0.5 / (7 * ((0.5 + a) / 0.25 + a / 0.125))
    visc = 0.5 / (49 * 0.1 * (16 + 64))
    src = 0.5 * 4.6 * 1e-3 / 1e3
    assert abs(orc.timestep(U, 0.5) - min(conv, visc, src)) < 1e-18



def _vdw_sound_speed(T, alpha, rho):
    """sqrt(p_alpha'(rho)) from the reduced Van-der-Waals pressure p = 8 T rho/(3 - rho) - 3 rho^2
    (Eq. vdw_p) and p_alpha = p + alpha rho^2/2 (Eq. modified_pressure), differentiated by hand."""
    return math.sqrt(24.0 * T / (3.0 - rho) ** 2 - 6.0 * rho + alpha * rho)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("nelem", [16, 24])
def test_parabolic_bound_is_the_printed_formula(N, nelem):
    """Eq. numerics_dfl prints dt <= CFL beta_RK(N) dxi^2 / (lambda^v (2N+1)^2) with
    lambda^v = max(eps, eps^2 gamma/beta) (Eq. numerics_nsk_visc_eigenvalues; here mu and kappa/beta).
    With beta_RK(N) folded into the CFL number (reading R9) and the parabolic bound the active one
    (fluid at rest, kappa/beta = 1 >> mu, mild alpha), the oracle's step is that formula on the
    element size h: a (2N+2) or (2N+1/2) offset misses it by 6% or more."""
    o = O.Oracle(1, (nelem,), (0,), (1,), N, alpha=2.0, beta=1.0, kappa=1.0, mu=1e-3)
    U = np.zeros(o.shape)
    U[0], U[2] = 2.1, 2.1
    h = 1.0 / nelem
    printed = 0.5 * h * h / (1.0 * (2 * N + 1) ** 2)
    conv = 0.5 * h / ((2 * N + 1) * _vdw_sound_speed(0.85, 2.0, 2.1))
    assert printed < conv and printed < 0.5 * 4.6 * 1.0 / 2.0  # the parabolic bound is the active one
    assert abs(o.timestep(U, 0.5) - printed) <= 1e-15 * printed


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_convective_bound_has_the_stated_scaling(N):
    """The convective bound (reading R9, the Cockburn-Shu CFL scaling of Runge-Kutta DG, which the
    paper leaves unstated) is dt = CFL h / ((2N+1) max(|v| + sqrt(p_alpha'))): with the convective
    bound active (inviscid limit, mild relaxation) the step times (2N+1) (|v| + a)/h equals the CFL
    number, on two element sizes; an offset other than 2N+1 changes the N-dependence."""
    for nelem in (12, 20):
        o = O.Oracle(1, (nelem,), (0,), (1,), N, alpha=10.0, beta=1.0, kappa=1e-8, mu=1e-8)
        U = np.zeros(o.shape)
        U[0], U[1], U[2] = 2.1, 2.1 * 0.4, 2.1
        lam = (0.4 + _vdw_sound_speed(0.85, 10.0, 2.1)) * nelem
        dt = o.timestep(U, 0.8)
        assert abs(dt * (2 * N + 1) * lam - 0.8) <= 1e-14


# ---------------------------------------------------------------- stress, numerical flux, symmetry

@pytest.mark.parametrize("model", [O.MODEL_RELAXATION, O.MODEL_NSK])
def test_shear_wave_residual_closed_form(model):
    """v = (A sin(2 pi y), 0) at uniform rho = c is an exact solution of both models: the flow is
    divergence-free, v . grad v = 0, the pressure, the Korteweg and relaxation terms are uniform,
    so only the shear stress acts, tau_xy = mu dv_x/dy (Eq. stress_nse) and
    d(rho v_x)/dt = mu d^2 v_x/dy^2 = -mu (2 pi)^2 A sin(2 pi y); every other residual is zero."""
    mu, A, rho0 = 5e-2, 0.3, 2.1
    errs = []
    for ne in (4, 8):  # alpha = 1 keeps the Lax-Friedrichs dissipation of the face jumps small
        o = O.Oracle(2, (ne, ne), (0, 0), (1, 1), 4, kappa=1e-4, alpha=1.0, beta=1e-3, mu=mu, model=model)
        y = o.coords()[1]
        U = np.zeros(o.shape)
        U[0] = rho0
        U[1] = rho0 * A * np.sin(2 * np.pi * y)
        if model == O.MODEL_RELAXATION:
            U[3] = rho0
        R = o.rhs(U)
        exact = -mu * (2 * np.pi) ** 2 * A * np.sin(2 * np.pi * y)
        scale = np.abs(exact).max()
        errs.append(np.abs(R[1] - exact).max() / scale)
        for v in [0, 2] + ([3] if model == O.MODEL_RELAXATION else []):
            assert np.abs(R[v]).max() < 1e-9 * scale, v
    assert errs[1] < 1e-2 and math.log2(errs[0] / errs[1]) > 3.0, errs


@pytest.mark.parametrize("dim,k", [(1, 0), (2, 0), (2, 1)])
def test_lax_friedrichs_coefficient_is_the_spectral_radius(dim, k):
    """The local Lax-Friedrichs flux of Sec. 3.1 dissipates with the larger of the two states'
    spectral radii of the convective flux Jacobian (its eigenvalues v_k and v_k +- sqrt(p_alpha'),
    Eq. parabolic_eigenvalues_model2). The Jacobian here is a central difference of the physical
    flux (the numerical flux of two equal states) and its eigenvalues come from numpy."""
    o = O.Oracle(dim, (2,) * dim, (0,) * dim, (1,) * dim, 2, alpha=10.0, beta=1e-3, kappa=1e-4, mu=1e-3)
    nv = dim + 2

    def state(rho, vel, c):
        return np.array([rho] + [rho * u for u in vel] + [c])

    UL = state(0.5, [0.3, -0.1][:dim], 0.55)
    UR = state(2.0, [-0.2, 0.25][:dim], 1.9)

    def flux(U):
        return o.numflux(k, U, U)

    def radius(U):
        n = nv - 1  # c has no convective flux
        J = np.zeros((n, n))
        for j in range(n):
            h = 1e-6 * max(1.0, abs(U[j]))
            Up, Um = U.copy(), U.copy()
            Up[j] += h
            Um[j] -= h
            J[:, j] = (flux(Up)[:n] - flux(Um)[:n]) / (2 * h)
        return np.abs(np.linalg.eigvals(J)).max()

    lam = max(radius(UL), radius(UR))
    assert abs(radius(UL) - radius(UR)) > 0.1 * lam  # the two states' radii differ clearly
    D = 0.5 * (flux(UL) + flux(UR)) - o.numflux(k, UL, UR)
    for v in range(nv - 1):  # rho and the momentum components
        assert abs(2 * D[v] / (UR[v] - UL[v]) - lam) < 1e-7 * lam, v
    assert abs(D[nv - 1]) < 1e-15  # no dissipation on c by default


@pytest.mark.parametrize("nt", [O.NODES_GAUSS, O.NODES_LOBATTO])
def test_mirror_symmetry_1d(nt):
    """x -> 1 - x (rho and c mirrored, momentum mirrored and negated) maps the residual the same
    way: the equations are reflection invariant and BR1 with central fluxes and the local
    Lax-Friedrichs flux keep that on a uniform mesh with symmetric nodes."""
    E, N = 8, 3
    o = O.Oracle(1, (E,), (0,), (1,), N, nt, alpha=100.0, beta=1e-2, kappa=1e-3, mu=2e-2)
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.2 * np.cos(4 * np.pi * x + 0.4)
    U[1] = U[0] * 0.1 * np.sin(2 * np.pi * x + 0.3)
    U[2] = U[0] * (1.0 + 0.01 * np.cos(2 * np.pi * x))

    def mirror(A):
        B = A[:, ::-1, ::-1].copy()
        B[1] = -B[1]
        return B

    R = o.rhs(U)
    Rm = o.rhs(mirror(U))
    for v in range(3):
        assert np.abs(Rm[v] - mirror(R)[v]).max() < 1e-11 * np.abs(R[v]).max(), v


# ---------------------------------------------------------------- time-step bounds and diagnostics

def _noise_after(o, U, dt, steps, v, ref):
    """max |U_v - ref| after the steps, inf where the state left the admissible range."""
    try:
        V = o.step(U, dt, steps)
    except O.OracleError:
        return math.inf
    return float(np.abs(V[v] - ref).max())


def test_source_bound_sits_at_the_real_axis_stability_limit():
    """dt_src = 4.6 beta/alpha (R9): the uniform relaxation c - rho ~ exp(-alpha t/beta) is one
    linear mode on the real axis, so one LSRK4 step multiplies c - rho by the scheme's stability
    function; it must not grow at the returned step and must grow 5% above it."""
    o = O.Oracle(1, (4,), (0,), (1,), 3, alpha=1e3, beta=1e-3, kappa=1e-4, mu=1e-3)
    U = np.zeros(o.shape)
    U[0], U[2] = 1.2, 1.25
    dt = o.timestep(U, 1.0)
    amp = lambda f: abs(o.step(U, f * dt, 1)[2][0, 0] - 1.2) / 0.05  # noqa: E731
    assert amp(1.0) <= 1.0 < amp(1.05)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_parabolic_bound_is_stable_and_not_vacuous(N):
    """Diffusion-dominated c (kappa/beta = 1 >> mu): grid-scale noise in c decays over 300 steps
    at the returned dt at CFL 0.5 (Eq. numerics_dfl with lambda^v = max(mu, kappa/beta) of
    Eq. visc_eigenvalues) and blows up at eight times that step (measured limits between CFL 0.5
    and 3 for N = 4..1)."""
    o = O.Oracle(1, (16,), (0,), (1,), N, alpha=1.0, beta=1e-3, kappa=1e-3, mu=1e-4)
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = 2.1
    U[2] = 2.1 + 1e-6 * np.random.default_rng(1).standard_normal(x.shape)
    dt = o.timestep(U, 0.5)
    assert _noise_after(o, U, dt, 300, 2, 2.1) < 1e-6
    assert _noise_after(o, U, 8.0 * dt, 300, 2, 2.1) > 1e-5


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_convective_bound_is_stable_and_not_vacuous(N):
    """Acoustics-dominated flow (mu, kappa ~ 0): noise in rho and m stays bounded over 600 steps
    at the returned dt at CFL 1 and blows up at three times that step (measured limits between
    CFL 1.25 and 2.5 for N = 4..1): the (2N+1) scaling of the bound tracks the DGSEM's spectral
    radius."""
    o = O.Oracle(1, (16,), (0,), (1,), N, alpha=10.0, beta=1.0, kappa=1e-8, mu=1e-8)
    x = o.coords()[0]
    rng = np.random.default_rng(2)
    U = np.zeros(o.shape)
    U[0] = 2.1 + 1e-6 * rng.standard_normal(x.shape)
    U[1] = 1e-6 * rng.standard_normal(x.shape)
    U[2] = 2.1
    dt = o.timestep(U, 1.0)
    assert _noise_after(o, U, dt, 600, 0, 2.1) < 1e-6
    assert _noise_after(o, U, 3.0 * dt, 600, 0, 2.1) > 1e-5


@pytest.mark.parametrize("dim", [1, 2])
def test_diagnostics_closed_forms(dim):
    """Mass, energy (Eq. pararelax_elliptical_energy_dynamic) and ||rho - c||_L2 of uniform rho,
    v and c = rho0 + A s(x) with s = sin(2 pi x) (1D) or sin(2 pi x) cos(2 pi y) (2D) on the
    unit box: mass = rho0, energy = rho0 |v|^2/2 + W(rho0) + alpha/2 A^2 <s^2> +
    kappa/2 (2 pi A)^2 <|grad s|^2/(2 pi)^2>, ||rho - c|| = A sqrt(<s^2>)."""
    rho0, A, alpha, kappa = 2.1, 0.05, 1.0, 1e-2
    vel = [0.5, -0.3][:dim]
    ne = (16,) if dim == 1 else (12, 10)
    o = O.Oracle(dim, ne, (0,) * dim, (1,) * dim, 4, alpha=alpha, beta=1e-3, kappa=kappa, mu=1e-3)
    X = o.coords()
    s = np.sin(2 * np.pi * X[0]) * (np.cos(2 * np.pi * X[1]) if dim == 2 else 1.0)
    U = np.zeros(o.shape)
    U[0] = rho0
    for a in range(dim):
        U[1 + a] = rho0 * vel[a]
    U[dim + 1] = rho0 + A * s
    s2, g2 = (0.5, 0.5) if dim == 1 else (0.25, 0.5)  # <s^2>, <|grad s|^2>/(2 pi)^2
    mass, energy, l2 = o.diagnostics(U)
    e_exact = (0.5 * rho0 * sum(u * u for u in vel) + O.free_energy(0.85, rho0) + 0.5 * alpha * A**2 * s2
               + 0.5 * kappa * (2 * np.pi * A) ** 2 * g2)
    assert abs(mass - rho0) < 1e-12
    assert abs(l2 - A * math.sqrt(s2)) < 1e-9 * A
    assert abs(energy - e_exact) < 1e-8 * abs(e_exact)
