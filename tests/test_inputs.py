"""The seeded input generators (paper_1912_12059_gb300/inputs.py) on the CPU: each recipe
against an independent fact (a numerical integral, the state it must describe, seeding)."""
import math

import numpy as np
import pytest

from paper_1912_12059_gb300 import inputs


def _grid_1d(n=20001):
    return np.linspace(0.0, 1.0, n)[None]


@pytest.mark.parametrize("kappa", [1e-4, 1e-3])
def test_gradient_theory_sigma_is_the_square_gradient_integral(kappa):
    """sigma = kappa * integral of rho'^2 over the tanh profile of width 2 sqrt(kappa): the
    closed form sqrt(kappa) (rho_l - rho_v)^2 / 6 against a trapezoidal integral."""
    rv, rl = inputs.PAPER_RHO_VAP, inputs.PAPER_RHO_LIQ
    w = inputs.interface_width(kappa)
    assert w == 2 * math.sqrt(kappa)
    x = np.linspace(-40 * w, 40 * w, 400001)
    drho = 0.5 * (rl - rv) / w / np.cosh(x / w) ** 2
    assert abs(kappa * np.trapezoid(drho**2, x) / inputs.gradient_theory_sigma(kappa) - 1.0) < 1e-8


def test_collision_velocity_reproduces_the_weber_number():
    kappa, r = 1e-4, 0.2
    for we in (10.0, 40.0, 80.0):
        v = inputs.collision_velocity(we, r, kappa)
        assert abs(2 * r * 1.0 * v * v / inputs.gradient_theory_sigma(kappa) - we) < 1e-10 * we


def test_slab_phases_and_symmetry():
    x = _grid_1d()
    U = inputs.slab_1d(x, kappa=1e-4)
    rho = U[0]
    i_mid, i_end = np.argmin(abs(x[0] - 0.5)), 0
    assert abs(rho[i_mid] - inputs.PAPER_RHO_LIQ) < 1e-9 and abs(rho[i_end] - inputs.PAPER_RHO_VAP) < 1e-9
    assert np.allclose(rho, rho[::-1], atol=1e-12)  # interfaces at 0.25 and 0.75
    assert np.all(U[1] == 0.0) and np.array_equal(U[2], rho)


def test_head_on_collision_drops_are_liquid_and_approach_each_other():
    g = np.linspace(0.0, 1.0, 41)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, 1, -1)
    v_rel = 0.8
    U = inputs.head_on_collision(X, v_rel, radius=0.2, kappa=1e-4)
    rho, mx = U[0, 0], U[1, 0]

    def at(p):
        return int(np.argmin(((X[:, 0, :].T - np.array(p)) ** 2).sum(axis=1)))

    left, right, far = at((0.25, 0.5, 0.5)), at((0.75, 0.5, 0.5)), at((0.5, 0.0, 0.0))
    assert abs(rho[left] - inputs.PAPER_RHO_LIQ) < 1e-6 and abs(rho[right] - inputs.PAPER_RHO_LIQ) < 1e-6
    assert abs(rho[far] - inputs.PAPER_RHO_VAP) < 1e-6
    v = mx / rho
    assert abs(v[left] - v_rel / 2) < 1e-6 and abs(v[right] + v_rel / 2) < 1e-6  # relative velocity v_rel
    assert abs(v[far]) < 1e-6
    assert np.all(U[2:4] == 0.0) and np.array_equal(U[4, 0], rho)


def test_droplets_mean_density_contour():
    """Sec. 4.2's n-droplet profile: liquid inside each drop, vapour outside, and the radius
    where rho crosses the mean (rho_v + rho_l)/2."""
    g = np.linspace(0.0, 1.0, 201)
    X = np.stack(np.meshgrid(g, g, indexing="ij")).reshape(2, 1, -1)
    U = inputs.droplets(X, [(0.3, 0.5), (0.72, 0.5)], [0.15, 0.1], kappa=1e-4)
    rho = U[0, 0].reshape(201, 201)
    mean = 0.5 * (inputs.PAPER_RHO_VAP + inputs.PAPER_RHO_LIQ)
    assert abs(rho[60, 100] - inputs.PAPER_RHO_LIQ) < 1e-6 and abs(rho[0, 0] - inputs.PAPER_RHO_VAP) < 1e-6
    row = rho[:, 100]  # along y = 0.5: the first drop spans x in (0.15, 0.45)
    i = np.where(np.diff((row > mean).astype(int)))[0]  # rho crosses the mean between g[i] and g[i+1]
    crossings = 0.5 * (g[i] + g[i + 1])
    assert abs(crossings[0] - 0.15) < 0.006 and abs(crossings[1] - 0.45) < 0.006


def test_riemann_states():
    x = np.array([[0.1, 0.49, 0.5, 0.9]])
    U = inputs.riemann_1d(x)
    assert list(U[0]) == [2.0, 2.0, 0.1, 0.1] and np.all(U[1] == 0.0) and np.array_equal(U[2], U[0])


def test_seeded_generators_are_reproducible_and_in_range():
    a = inputs.random_state((4, 7, 16), seed=3)
    b = inputs.random_state((4, 7, 16), seed=3)
    c = inputs.random_state((4, 7, 16), seed=4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a[0].min() >= 1.0 and a[0].max() <= 1.4
    assert np.abs(a[1:3] / a[0]).max() <= 0.2 + 1e-15
    assert np.abs(a[3] / a[0] - 1.0).max() <= 0.02 + 1e-15
    U = inputs.slab_1d(_grid_1d(101))
    n1, n2 = inputs.add_density_noise(U, 1e-4, seed=5), inputs.add_density_noise(U, 1e-4, seed=5)
    assert np.array_equal(n1, n2) and 0 < np.abs(n1[0] - U[0]).max() <= 1e-4 and np.array_equal(n1[-1], n1[0])
