"""Pins of the oracle's HLLC flux for model II (the three-wave solver of Toro's textbook, which
Sec. 3.1 refers to, applied to the barotropic system (rho, m) with the modified pressure
p_alpha; c is not transported). Each test checks a property that the mathematics of the
solver fixes, independently of how the oracle writes it:

* consistency: equal states give the physical flux;
* upwinding: when every wave moves one way the flux is that side's physical flux;
* contact resolution: a stationary shear layer (equal rho, zero normal velocity, different
  tangential velocity) is an exact steady solution, so its flux carries no tangential
  momentum (local Lax-Friedrichs smears it); a moving one takes the upwind tangential momentum;
* mirror symmetry of the normal direction;
* the residual with HLLC preserves free streams, conserves mass, reaches the design order on a
  manufactured solution and lets the energy decay.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs

T, ALPHA = 0.85, 1e3


def _orc(dim=3, flux=O.FLUX_HLLC):
    return O.Oracle(dim, (2,) * dim, (0,) * dim, (1,) * dim, 3, flux=flux, T=T, alpha=ALPHA)


def _p_alpha(rho):
    return O.pressure(T, rho) + 0.5 * ALPHA * rho * rho


def _a(rho):
    return math.sqrt(O.dpressure(T, rho) + ALPHA * rho)


def _phys_flux(U, k, dim=3):
    rho = U[0]
    f = np.zeros(dim + 2)
    f[0] = U[1 + k]
    for a in range(dim):
        f[1 + a] = U[1 + k] * U[1 + a] / rho
    f[1 + k] += _p_alpha(rho)
    return f


def _state(rho, v, c=None):
    v = np.asarray(v, dtype=float)
    return np.concatenate([[rho], rho * v, [rho if c is None else c]])


@pytest.mark.parametrize("k", [0, 1, 2])
def test_consistency(k):
    o = _orc()
    rng = np.random.default_rng(k)
    for _ in range(5):
        U = _state(rng.uniform(0.4, 2.2), rng.uniform(-3, 3, 3), rng.uniform(0.5, 2.0))
        F = o.numflux(k, U, U)
        assert np.allclose(F, _phys_flux(U, k), rtol=1e-14, atol=1e-12)


def test_supersonic_upwinding():
    o = _orc()
    rl, rr = 1.1, 1.5
    ul = _a(rl) + 5.0   # u - a > 0 on both sides: all waves move right
    ur = _a(rr) + 4.0
    UL, UR = _state(rl, [ul, 0.3, -0.2]), _state(rr, [ur, -0.1, 0.4])
    assert np.allclose(o.numflux(0, UL, UR), _phys_flux(UL, 0), rtol=1e-14, atol=1e-12)
    UL, UR = _state(rl, [-ul, 0.3, -0.2]), _state(rr, [-ur, -0.1, 0.4])  # all waves move left
    assert np.allclose(o.numflux(0, UL, UR), _phys_flux(UR, 0), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_stationary_shear_layer_is_exact(k):
    rho = 1.3
    vl, vr = np.array([0.4, -0.7, 0.2]), np.array([-0.5, 0.6, 0.9])
    vl[k] = vr[k] = 0.0
    UL, UR = _state(rho, vl), _state(rho, vr)
    F = _orc().numflux(k, UL, UR)
    want = np.zeros(5)
    want[1 + k] = _p_alpha(rho)
    assert np.allclose(F, want, rtol=1e-14, atol=1e-12)
    # local Lax-Friedrichs dissipates the tangential jump
    Flf = _orc(flux=O.FLUX_LF).numflux(k, UL, UR)
    t = [a for a in range(3) if a != k][0]
    assert abs(Flf[1 + t]) > 0.1


def test_moving_shear_layer_takes_upwind_tangential_momentum():
    rho, u = 1.3, 0.8  # subsonic (a ~ 36): the contact moves right at u
    UL, UR = _state(rho, [u, 0.4, -0.3]), _state(rho, [u, -0.6, 0.9])
    F = _orc().numflux(0, UL, UR)
    assert np.allclose(F[:2], [rho * u, rho * u * u + _p_alpha(rho)], rtol=1e-13)
    assert np.allclose(F[2:4], rho * u * np.array([0.4, -0.3]), rtol=1e-12, atol=1e-13)
    UL, UR = _state(rho, [-u, 0.4, -0.3]), _state(rho, [-u, -0.6, 0.9])  # moving left
    F = _orc().numflux(0, UL, UR)
    assert np.allclose(F[2:4], -rho * u * np.array([-0.6, 0.9]), rtol=1e-12, atol=1e-13)


def test_no_convective_flux_of_c():
    o = _orc()
    F = o.numflux(1, _state(0.5, [0.1, 2.0, 0.3], c=0.9), _state(1.9, [-0.4, -1.0, 0.2], c=1.4))
    assert F[4] == 0.0


def test_mirror_symmetry():
    """Reflecting the normal direction swaps the states: the mass flux changes sign, the normal
    momentum flux is unchanged and the tangential momentum fluxes change sign."""
    o = _orc()
    rng = np.random.default_rng(5)
    for _ in range(10):
        UL = _state(rng.uniform(0.4, 2.2), rng.uniform(-30, 30, 3))
        UR = _state(rng.uniform(0.4, 2.2), rng.uniform(-30, 30, 3))
        F = o.numflux(0, UL, UR)
        mL, mR = UL.copy(), UR.copy()
        mL[1] *= -1
        mR[1] *= -1
        G = o.numflux(0, mR, mL)
        scale = np.abs(F).max()
        assert abs(F[0] + G[0]) < 1e-13 * scale
        assert abs(F[1] - G[1]) < 1e-13 * scale
        assert np.all(np.abs(F[2:4] + G[2:4]) < 1e-13 * scale)


def test_residual_free_stream_and_mass_conservation():
    o = O.Oracle(3, (3, 2, 2), (0, 0, 0), (1.0, 0.7, 1.3), 3, flux=O.FLUX_HLLC)
    U = np.zeros(o.shape)
    U[0] = 1.3
    U[1], U[2], U[3] = 0.5, -0.2, 0.1
    U[4] = 1.3
    assert np.abs(o.rhs(U)).max() < 1e-13 * 1e3 * 3 * 16
    o = O.Oracle(2, (4, 3), (0, 0), (1, 1), 3, flux=O.FLUX_HLLC, alpha=50.0, beta=0.05, kappa=1e-3, mu=1e-2)
    U = inputs.random_state(o.shape, seed=12)
    m0 = o.diagnostics(U)[0]
    R = o.rhs(U)
    wq = np.ones(o.npe)  # quadrature weights of the reference element (uniform mesh: J is common)
    for n in range(o.npe):
        wq[n] = o.w[n % o.np] * o.w[n // o.np]
    assert abs((R[0] * wq).sum()) < 1e-13 * np.abs(R[0] * wq).sum()
    assert abs(o.diagnostics(o.step(U, 1e-5, 3))[0] - m0) < 1e-13 * abs(m0)


def test_energy_decay_static_interface_hllc():
    rv, rl, _ = O.maxwell(0.85)
    orc = O.Oracle(1, (24,), (0,), (1,), 3, O.NODES_GAUSS, alpha=100.0, beta=1e-2, kappa=4e-4, mu=1e-2,
                   flux=O.FLUX_HLLC)
    U = inputs.slab_1d(orc.coords(), rv, rl, kappa=4e-4)
    dt = orc.timestep(U, 0.5)
    energies = [orc.diagnostics(U)[1]]
    for _ in range(20):
        U = orc.step(U, dt, 5)
        energies.append(orc.diagnostics(U)[1])
    assert (np.diff(energies) <= 1e-12 * abs(energies[0])).all()
    assert energies[-1] < energies[0]
