"""Pins of the oracle's finite-volume sub-cell shock capturing (Sec. 3.2, the sub-cell section)
and its Dirichlet boundaries (the 1D sharp-interface Riemann problem of Sec. 4). No GPU.

Each check rests on something other than the oracle's own formulas: exact integrals of
monomials, the orthonormality of the Legendre modes, the existing (separately pinned) DG
residual, free-stream states, telescoping fluxes (conservation), the exactness of the
MinMod-limited linear reconstruction for linear data, and the exactness of centred
differences of cell means for a quadratic.
"""
import numpy as np
import pytest

import oracle as O

PRM = dict(T=0.85, kappa=1e-4, alpha=100.0, beta=1e-3, mu=1e-3)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("node_type", [O.NODES_GAUSS, O.NODES_LOBATTO])
def test_subcell_means_are_exact_integrals(N, node_type):
    """M maps the nodal values of xi^k (k <= N) to the exact means over the N+1 equal sub-cells."""
    M, Minv = O.fv_tables(N, node_type)
    xi, _ = O.nodes(N, node_type)
    np_ = N + 1
    edges = -1.0 + 2.0 * np.arange(np_ + 1) / np_
    for k in range(N + 1):
        exact = (edges[1:] ** (k + 1) - edges[:-1] ** (k + 1)) / (k + 1) / (2.0 / np_)
        assert np.allclose(M @ xi**k, exact, rtol=0, atol=1e-13), k
    assert np.allclose(Minv @ M, np.eye(np_), atol=1e-12)


@pytest.mark.parametrize("N", [2, 3, 4, 6])
@pytest.mark.parametrize("node_type", [O.NODES_GAUSS, O.NODES_LOBATTO])
def test_persson_indicator_closed_forms(N, node_type):
    """Ind = log10 of the top orthonormal mode's energy share: -inf for a constant, 0 for the
    top mode alone, log10(b^2 / (a^2 + b^2)) for a phi_1 + b phi_N (phi_m = sqrt((2m+1)/2) P_m)."""
    xi, _ = O.nodes(N, node_type)
    phi = lambda m: np.sqrt((2 * m + 1) / 2.0) * np.polynomial.legendre.legval(xi, [0] * m + [1])  # noqa: E731
    assert O.persson(np.full(N + 1, 1.7), node_type) < -25.0
    assert abs(O.persson(phi(N), node_type)) < 1e-12
    for a, b in ((1.0, 1e-3), (2.0, 0.5), (0.3, 1.0)):
        got = O.persson(a * phi(1) + b * phi(N), node_type)
        assert abs(got - np.log10(b * b / (a * a + b * b))) < 1e-10, (a, b)


def _smooth_state(o, dirichlet=False):
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = 1.0 + 0.3 * np.sin(2 * np.pi * x)
    U[1] = 0.1 * np.cos(2 * np.pi * x) * U[0]
    U[2] = U[0] + 0.01 * np.sin(4 * np.pi * x)
    return U


def _to_means(U, flags, N, node_type=O.NODES_GAUSS):
    M, _ = O.fv_tables(N, node_type)
    V = U.copy()
    for e in np.nonzero(flags)[0]:
        for v in range(U.shape[0]):
            V[v, e] = M @ U[v, e]
    return V


@pytest.mark.parametrize("flux", [O.FLUX_LF, O.FLUX_HLLC])
def test_all_dg_periodic_equals_the_dg_residual(flux):
    o = O.Oracle(1, (10,), (0.0,), (1.0,), 3, flux=flux, **PRM)
    o.fv_setup(dirichlet=False)
    U = _smooth_state(o)
    R = o.rhs(U)
    assert np.abs(o.fv_rhs(U, np.zeros(o.E, np.int32)) - R).max() <= 1e-13 * np.abs(R).max()


@pytest.mark.parametrize("pattern", ["dg", "mixed", "fv"])
@pytest.mark.parametrize("flux", [O.FLUX_LF, O.FLUX_HLLC])
def test_free_stream_with_dirichlet_boundaries(pattern, flux):
    """A constant state equal to both boundary states is steady on any DG/FV pattern."""
    o = O.Oracle(1, (9,), (0.0,), (1.0,), 3, flux=flux, **PRM)
    Ub = (1.2, 0.15, 1.2)
    o.fv_setup(dirichlet=True, Ub_lo=Ub, Ub_hi=Ub)
    flags = {"dg": np.zeros(9), "fv": np.ones(9), "mixed": np.arange(9) % 2}[pattern].astype(np.int32)
    U = np.zeros(o.shape)
    for v in range(3):
        U[v] = Ub[v]
    assert np.abs(o.fv_rhs(U, flags)).max() < 1e-10


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("flux", [O.FLUX_LF, O.FLUX_HLLC])
def test_mass_and_momentum_conservation_on_a_mixed_periodic_mesh(N, flux):
    """Shared face fluxes telescope: with periodic boundaries the total mass changes at a
    rate of zero (DG: Gauss quadrature of the residual; FV: sub-cell means times width)."""
    E = 12
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, flux=flux, **PRM)
    o.fv_setup(dirichlet=False)
    flags = ((np.arange(E) % 3) == 1).astype(np.int32)
    U = _to_means(_smooth_state(o), flags, N)
    R = o.fv_rhs(U, flags)
    h = 1.0 / E
    _, w = O.nodes(N)
    rate = sum((R[0, e].sum() * h / (N + 1)) if flags[e] else (R[0, e] * w * h / 2).sum() for e in range(E))
    assert abs(rate) < 1e-14 * np.abs(R[0]).max()


@pytest.mark.parametrize("flux", [O.FLUX_LF, O.FLUX_HLLC])
@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("ends", [(0.6, 1.9, 0.7, 1.6), (1.9, 0.6, 1.6, 0.7)], ids=["rising", "falling"])
def test_fv_residual_is_exact_for_linear_data(flux, N, ends):
    """rho and c linear, v = 0, every element FV, Dirichlet states equal to the exact boundary
    values: MinMod returns the exact slope, the reconstruction is exact, both face states agree,
    so each cell's residual equals the exact cell average of the right-hand side:
      rho: 0;  m: -(p_alpha(rho(x+)) - p_alpha(rho(x-))) / dx + alpha rho_mean c_x;
      c: (alpha / beta) (rho_mean - c_mean)  (the diffusive fluxes are constant and cancel)."""
    E = 7
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, flux=flux, **PRM)
    r0, r1, c0, c1 = ends
    o.fv_setup(dirichlet=True, Ub_lo=(r0, 0.0, c0), Ub_hi=(r1, 0.0, c1))
    nc = E * (N + 1)
    dx = 1.0 / nc
    edges = np.arange(nc + 1) * dx
    mid = 0.5 * (edges[1:] + edges[:-1])
    rho, c = r0 + (r1 - r0) * mid, c0 + (c1 - c0) * mid
    U = np.zeros(o.shape)
    U[0] = rho.reshape(E, N + 1)
    U[2] = c.reshape(E, N + 1)
    R = o.fv_rhs(U, np.ones(E, np.int32))
    pa = lambda r: O.pressure(PRM["T"], r) + PRM["alpha"] * r * r / 2  # noqa: E731
    rho_e = r0 + (r1 - r0) * edges
    exact_m = -(np.array([pa(r) for r in rho_e[1:]]) - np.array([pa(r) for r in rho_e[:-1]])) / dx
    exact_m += PRM["alpha"] * rho * (c1 - c0)
    exact_c = PRM["alpha"] / PRM["beta"] * (rho - c)
    assert np.abs(R[0]).max() < 1e-9
    assert np.allclose(R[1].ravel(), exact_m, rtol=1e-11, atol=1e-9)
    assert np.allclose(R[2].ravel(), exact_c, rtol=1e-11, atol=1e-7)


def test_switching_conserves_mass_and_flags_the_jump():
    """An element holding a jump switches to FV (Ind above the upper threshold), smooth ones
    stay DG; each switch keeps the element's integral; back-switching needs Ind below the
    lower threshold (hysteresis)."""
    N, E = 3, 8
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, **PRM)
    o.fv_setup(dirichlet=True, Ub_lo=(2.0, 0, 2.0), Ub_hi=(0.1, 0, 0.1))
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = np.where(x < 0.55, 2.0, 0.1)  # the jump inside element 4 (0.5 .. 0.625)
    U[2] = U[0]
    _, w = O.nodes(N)
    h = 1.0 / E
    mass = lambda V, f: sum(  # noqa: E731
        (V[0, e].sum() * h / (N + 1)) if f[e] else (V[0, e] * w * h / 2).sum() for e in range(E))
    U2, f2, ind = o.fv_switch(U, np.zeros(E, np.int32))
    assert list(f2) == [0, 0, 0, 0, 1, 0, 0, 0]
    assert ind[4] > -6 and all(ind[e] < -25 for e in range(E) if e != 4)
    assert abs(mass(U2, f2) - mass(U, np.zeros(E))) < 1e-14
    # the sub-cell means of the element with the jump: mean of the nodal polynomial
    M, _ = O.fv_tables(N)
    assert np.allclose(U2[0, 4], M @ U[0, 4], atol=1e-15)
    # hysteresis: thresholds that put this element's Ind between lower and upper keep it FV
    o.fv_setup(dirichlet=True, Ub_lo=(2.0, 0, 2.0), Ub_hi=(0.1, 0, 0.1), ind_upper=ind[4] + 1.0,
               ind_lower=-30.0)
    U3, f3, _ = o.fv_switch(U2, f2)
    assert list(f3) == list(f2) and np.array_equal(U3, U2)
    # a smooth FV element returns to DG with its polynomial recovered exactly
    f4 = np.zeros(E, np.int32)
    f4[1] = 1
    V = _to_means(U, f4, N)
    o.fv_setup(dirichlet=True, Ub_lo=(2.0, 0, 2.0), Ub_hi=(0.1, 0, 0.1))
    U5, f5, _ = o.fv_switch(V, f4)
    assert f5[1] == 0 and np.allclose(U5[:, 1], U[:, 1], atol=1e-13)


def test_sharp_interface_riemann_problem_runs_bounded():
    """The Riemann problem of Sec. 4 (liquid 2.0 | vapour 0.1, alpha 100, beta 1e-3, HLLC,
    Persson thresholds -6 / -8, Dirichlet boundaries, CFL 0.1) on 40 elements, N = 3: the
    elements next to the discontinuity switch to FV, the density stays inside (0, 3) and the
    total mass changes only through the boundary fluxes (which vanish while the waves have not
    reached the boundaries)."""
    N, E = 3, 40
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, flux=O.FLUX_HLLC, T=0.85, kappa=1e-6, alpha=100.0, beta=1e-3,
                 mu=1e-3)
    o.fv_setup(dirichlet=True, Ub_lo=(2.0, 0, 2.0), Ub_hi=(0.1, 0, 0.1))
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = np.where(x < 0.5, 2.0, 0.1)
    U[2] = U[0]
    dt = o.timestep(U, 0.1)
    flags = np.zeros(E, np.int32)
    _, w = O.nodes(N)
    h = 1.0 / E
    m0 = (U[0] * w * h / 2).sum()
    U, flags = o.fv_step(U, flags, dt, 60)
    assert flags.sum() >= 1 and flags[:10].sum() == 0 and flags[-10:].sum() == 0
    assert np.all(U[0] > 0.05) and np.all(U[0] < 2.3)
    m1 = sum((U[0, e].sum() * h / (N + 1)) if flags[e] else (U[0, e] * w * h / 2).sum() for e in range(E))
    assert abs(m1 - m0) < 1e-12 * m0


@pytest.mark.parametrize("N", [2, 3])
def test_fv_source_and_diffusion_exact_for_quadratic_c(N):
    """rho constant, v = 0, c quadratic, every element FV. Centred differences of the cell means
    of a quadratic are exact, so in the interior cells (away from the half-width boundary
    quotients) the momentum residual is alpha rho c'(x_j) (the source's c_x is the mean of the
    two face quotients) and the c residual is (kappa/beta) c'' + (alpha/beta)(rho - c_mean)."""
    E = 6
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, **PRM)
    rho, a, b, q = 1.3, 0.9, 0.4, 0.5  # c = a + b x + q x^2
    o.fv_setup(dirichlet=True, Ub_lo=(rho, 0.0, a), Ub_hi=(rho, 0.0, a + b + q))
    nc = E * (N + 1)
    dx = 1.0 / nc
    xl = np.arange(nc) * dx
    xr = xl + dx
    cmean = a + b * (xl + xr) / 2 + q * (xr**3 - xl**3) / (3 * dx)
    U = np.zeros(o.shape)
    U[0] = rho
    U[2] = cmean.reshape(E, N + 1)
    R = o.fv_rhs(U, np.ones(E, np.int32))
    mid = 0.5 * (xl + xr)
    inner = slice(1, nc - 1)
    exact_m = PRM["alpha"] * rho * (b + 2 * q * mid)
    exact_c = PRM["kappa"] / PRM["beta"] * 2 * q + PRM["alpha"] / PRM["beta"] * (rho - cmean)
    assert np.abs(R[0]).max() < 1e-9
    assert np.allclose(R[1].ravel()[inner], exact_m[inner], rtol=1e-10, atol=1e-8)
    assert np.allclose(R[2].ravel()[inner], exact_c[inner], rtol=1e-10, atol=1e-6)


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("node_type", [O.NODES_GAUSS, O.NODES_LOBATTO])
def test_fv_element_holding_a_polynomial_switches_back_exactly(N, node_type):
    """An FV element whose sub-cell means are those of a polynomial of degree below N (exact
    integrals of monomials, not the oracle's mean matrix) is smooth: its indicator is that of the
    polynomial's nodal values (no top mode), it switches back to DG and the conversion returns
    the polynomial's nodal values."""
    E = 5
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, node_type, **PRM)
    o.fv_setup()
    xi, _ = O.nodes(N, node_type)
    np_ = N + 1
    edges = -1.0 + 2.0 * np.arange(np_ + 1) / np_
    coef = {0: (1.2, 0.3, -0.2), 1: (0.1, -0.05, 0.02), 2: (1.25, 0.2, 0.1)}  # rho, m, c in xi
    U = np.zeros(o.shape)
    for v, (a0, a1, a2) in coef.items():
        U[v] = a0  # the DG elements: constant states
        poly = lambda t: a0 + a1 * t + (a2 * t * t if N > 2 else 0.0)  # noqa: E731
        mean = [a0 + a1 * (edges[j + 1] ** 2 - edges[j] ** 2) / 2 / (edges[j + 1] - edges[j])
                + ((a2 * (edges[j + 1] ** 3 - edges[j] ** 3) / 3 / (edges[j + 1] - edges[j])) if N > 2 else 0.0)
                for j in range(np_)]
        U[v, 2] = mean
        coef[v] = poly(xi)
    flags = np.zeros(E, np.int32)
    flags[2] = 1
    U2, f2, ind = o.fv_switch(U, flags)
    assert ind[2] < -25.0 and O.persson(coef[0], node_type) < -25.0, ind  # both at round-off: no top mode
    assert list(f2) == [0] * E
    for v in range(3):
        assert np.allclose(U2[v, 2], coef[v], rtol=0, atol=1e-13), v


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("pattern", [(0, 1, 1, 0, 1, 0, 0), (1, 0, 1, 1, 0, 0, 1)])
def test_mixed_mesh_exact_for_linear_c(N, pattern):
    """rho constant, v = 0, c linear, DG and FV elements mixed, Dirichlet states equal to the
    exact boundary values: the lifted gradient (DG) and every face quotient (FV, across FV-FV,
    DG-FV and boundary faces) equal the slope, so the diffusive fluxes are equal on both sides of
    every face and cancel: R_rho = 0, R_m = alpha rho c_x and R_c = (alpha/beta)(rho - c) in every
    DG node and FV sub-cell."""
    E = len(pattern)
    flags = np.array(pattern, np.int32)
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, **PRM)
    rho, a, b = 1.3, 0.9, 0.6  # c = a + b x
    o.fv_setup(dirichlet=True, Ub_lo=(rho, 0.0, a), Ub_hi=(rho, 0.0, a + b))
    xn = o.coords()[0]
    h, dx = 1.0 / E, 1.0 / (E * (N + 1))
    U = np.zeros(o.shape)
    U[0] = rho
    for e in range(E):
        U[2, e] = (a + b * (e * h + (np.arange(N + 1) + 0.5) * dx)) if flags[e] else (a + b * xn[e])
    R = o.fv_rhs(U, flags)
    assert np.abs(R[0]).max() < 1e-9
    assert np.allclose(R[1], PRM["alpha"] * rho * b, rtol=1e-10, atol=1e-8)
    assert np.allclose(R[2], PRM["alpha"] / PRM["beta"] * (rho - U[2]), rtol=1e-10, atol=1e-6)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_dirichlet_dg_exact_for_quadratic_c(N):
    """rho constant, v = 0, c quadratic, every element DG, Dirichlet states equal to the exact
    boundary values: BR1 is exact for polynomials of degree <= N, and the boundary face's viscous
    flux takes the interior side's gradient at that face, so every node, the boundary elements
    included, has R_m = alpha rho c'(x) and R_c = (kappa/beta) c'' + (alpha/beta)(rho - c)."""
    E = 5
    o = O.Oracle(1, (E,), (0.0,), (1.0,), N, **PRM)
    rho, a, b, q = 1.3, 0.9, 0.4, 0.5  # c = a + b x + q x^2
    o.fv_setup(dirichlet=True, Ub_lo=(rho, 0.0, a), Ub_hi=(rho, 0.0, a + b + q))
    x = o.coords()[0]
    U = np.zeros(o.shape)
    U[0] = rho
    U[2] = a + b * x + q * x * x
    R = o.fv_rhs(U, np.zeros(E, np.int32))
    assert np.abs(R[0]).max() < 1e-9
    assert np.allclose(R[1], PRM["alpha"] * rho * (b + 2 * q * x), rtol=1e-10, atol=1e-8)
    exact_c = PRM["kappa"] / PRM["beta"] * 2 * q + PRM["alpha"] / PRM["beta"] * (rho - U[2])
    assert np.allclose(R[2], exact_c, rtol=1e-10, atol=1e-6)
