"""Seeded synthetic initial conditions for the relaxation-model workloads.

This module holds no arithmetic of the discretisation: every function takes the
physical node coordinates (from `Solver.node_coords()` or any equivalent) and
returns the state in the canonical layout [nvar][E][npe] with variables
(rho, rho v_1..rho v_dim, c). Random draws use numpy's PCG64 with an explicit
seed. Phase densities are arguments; the defaults are the saturation densities
the paper prints at T = 0.85 (Sec. 4.1.1: rho_vap = 0.3197, rho_liq = 1.8071).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PAPER_RHO_VAP = 0.3197
PAPER_RHO_LIQ = 1.8071
SEED = 20191226


def interface_width(kappa: float) -> float:
    """Width parameter 2 sqrt(kappa) of the tanh profiles of Sec. 4 (kappa = eps^2 gamma)."""
    return 2.0 * math.sqrt(kappa)


def _pack(rho, mom, c):
    return np.ascontiguousarray(np.stack([rho, *mom, c]), dtype=np.float64)


def slab_1d(x, rho_vap=PAPER_RHO_VAP, rho_liq=PAPER_RHO_LIQ, kappa=1e-4, x0=0.25, x1=0.75):
    """Static liquid slab on a periodic interval: two tanh interfaces at x0 and x1
    (the static profile of Sec. 4.1.1 made periodic), v = 0, c = rho."""
    x = x[0]
    wd = interface_width(kappa)
    rho = rho_vap + 0.5 * (rho_liq - rho_vap) * (np.tanh((x - x0) / wd) - np.tanh((x - x1) / wd))
    return _pack(rho, [np.zeros_like(rho)], rho.copy())


def droplets(x, centres, radii, rho_vap=PAPER_RHO_VAP, rho_liq=PAPER_RHO_LIQ, kappa=1e-4):
    """n droplets at rest, Sec. 4.2 Eq. (results_nsk_2d_merge_initialcondition):
    rho = (n rho_l - (n-2) rho_v)/2 + sum_i (rho_v - rho_l)/2 tanh((d_i - r_i)/(2 sqrt(kappa)))."""
    n = len(radii)
    wd = interface_width(kappa)
    rho = np.full(x.shape[1:], 0.5 * (n * rho_liq - (n - 2) * rho_vap))
    for c0, r in zip(centres, radii):
        d = np.sqrt(sum((x[k] - c0[k]) ** 2 for k in range(x.shape[0])))
        rho = rho + 0.5 * (rho_vap - rho_liq) * np.tanh((d - r) / wd)
    return _pack(rho, [np.zeros_like(rho) for _ in range(x.shape[0])], rho.copy())


def head_on_collision(x, v_rel, radius=0.2, centres=((0.25, 0.5, 0.5), (0.75, 0.5, 0.5)),
                      rho_vap=PAPER_RHO_VAP, rho_liq=PAPER_RHO_LIQ, kappa=1e-4, split=0.5):
    """Two droplets moving toward each other along x, Sec. 4.3 Eq. (hoc_initialcondition),
    with the liquid inside the drops (1 - tanh) and the x-velocity profile of the paper:
    v_1 = +-v_rel/4 (1 - tanh((d_i - r)/(2 sqrt(kappa)))) left / right of x = split."""
    wd = interface_width(kappa)
    dist = []
    rho = np.full(x.shape[1:], rho_vap)
    for c0 in centres:
        d = np.sqrt(sum((x[k] - c0[k]) ** 2 for k in range(x.shape[0])))
        dist.append(d)
        rho = rho + 0.5 * (rho_liq - rho_vap) * (1.0 - np.tanh((d - radius) / wd))
    v1 = np.where(x[0] < split,
                  0.25 * v_rel * (1.0 - np.tanh((dist[0] - radius) / wd)),
                  -0.25 * v_rel * (1.0 - np.tanh((dist[1] - radius) / wd)))
    mom = [rho * v1] + [np.zeros_like(rho) for _ in range(x.shape[0] - 1)]
    return _pack(rho, mom, rho.copy())


def riemann_1d(x, rho_left=2.0, rho_right=0.1, x0=0.5):
    """Multiphase shock tube of Sec. 4 (sharp-interface limit): liquid rho_left at rest left of
    x0, vapour rho_right at rest right of it, c = rho (a node exactly at x0 takes the right
    state)."""
    x = x[0]
    rho = np.where(x < x0, rho_left, rho_right).astype(np.float64)
    return _pack(rho, [np.zeros_like(rho)], rho.copy())


def gradient_theory_sigma(kappa, rho_vap=PAPER_RHO_VAP, rho_liq=PAPER_RHO_LIQ):
    """Surface tension kappa * integral(rho'^2) of the tanh profile of width 2 sqrt(kappa):
    sqrt(kappa) (rho_l - rho_v)^2 / 6 (square-gradient theory; the paper fixes no value)."""
    return math.sqrt(kappa) * (rho_liq - rho_vap) ** 2 / 6.0


def collision_velocity(we, radius, kappa, rho_vap=PAPER_RHO_VAP, rho_liq=PAPER_RHO_LIQ, rho_c=1.0):
    """Relative velocity for collision Weber number We = 2 r rho_c v_rel^2 / sigma (Sec. 4.3,
    Eq. results_nsk_weber_collision read with v_rel squared, which reproduces the HOC table)."""
    sigma = gradient_theory_sigma(kappa, rho_vap, rho_liq)
    return math.sqrt(we * sigma / (2.0 * radius * rho_c))


def add_density_noise(U, amplitude, seed=SEED):
    """Uniform white noise in [-amplitude, amplitude] on rho (seeded PCG64), then c = rho."""
    rng = np.random.Generator(np.random.PCG64(seed))
    U = U.copy()
    U[0] += rng.uniform(-amplitude, amplitude, size=U[0].shape)
    U[-1] = U[0]
    return U


def random_state(shape_nvar_E_npe, seed=SEED, rho_range=(1.0, 1.4), v_amp=0.2, c_amp=0.02):
    """Random in-range state for operator tests: rho uniform in rho_range, v uniform in
    [-v_amp, v_amp], c = rho (1 + uniform(-c_amp, c_amp))."""
    nvar, E, npe = shape_nvar_E_npe
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.uniform(*rho_range, size=(E, npe))
    vel = [rng.uniform(-v_amp, v_amp, size=(E, npe)) for _ in range(nvar - 2)]
    c = rho * (1.0 + rng.uniform(-c_amp, c_amp, size=(E, npe)))
    return _pack(rho, [rho * v for v in vel], c)


# ---------------------------------------------------------------------------
# Named workloads (mesh + parameters + initial condition recipe)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    dim: int
    nelem: tuple
    N: int
    node_type: int = 0  # 0 Gauss-Legendre, 1 Gauss-Lobatto
    T: float = 0.85
    kappa: float = 1e-4
    alpha: float = 1e3
    beta: float = 1e-3
    mu: float = 1e-3
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    cfl: float = 0.5
    steps: int = 100
    extra: dict = field(default_factory=dict)

    @property
    def npe(self):
        return (self.N + 1) ** self.dim

    @property
    def n_elem(self):
        return int(np.prod(self.nelem))

    @property
    def dofs(self):
        return self.n_elem * self.npe

    def initial_state(self, x, rho_vap=PAPER_RHO_VAP, rho_liq=PAPER_RHO_LIQ):
        """State on node coordinates x[dim][E][npe]."""
        kind = self.extra.get("ic", "")
        if kind == "slab":
            return slab_1d(x, rho_vap, rho_liq, self.kappa)
        if kind == "droplets":
            U = droplets(x, self.extra["centres"], self.extra["radii"], rho_vap, rho_liq, self.kappa)
            amp = self.extra.get("noise", 0.0)
            return add_density_noise(U, amp, self.extra.get("seed", SEED)) if amp else U
        if kind == "collision":
            v_rel = collision_velocity(self.extra["we"], self.extra["radius"], self.kappa, rho_vap, rho_liq)
            c = self.extra.get("centres", ((0.25, 0.5, 0.5), (0.75, 0.5, 0.5)))
            return head_on_collision(x, v_rel, self.extra["radius"], c, rho_vap, rho_liq, self.kappa)
        if kind == "riemann":
            return riemann_1d(x, self.extra["rho_left"], self.extra["rho_right"], self.extra.get("x0", 0.5))
        raise ValueError(f"unknown initial condition {kind!r}")


def static_interface_1d(N=3, node_type=1, nelem=64):
    """1D static phase interface: periodic [0,1], 64 elements, N=3 Gauss-Lobatto,
    kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3, LSRK4 2000 steps at CFL 0.5."""
    return Workload("static_interface_1d_E64_N3", 1, (nelem,), N, node_type, steps=2000,
                    extra={"ic": "slab"})


def riemann_1d_sharp(eps=1e-3, nelem=200, N=3, gamma=1.0):
    """1D multiphase Riemann problem in the sharp-interface limit (Sec. 4): (0, 1), 200 elements,
    N = 3, liquid 2.0 | vapour 0.1 at rest (c = rho), alpha = 100, beta = 1e-3, capillarity
    gamma = 1, viscosity mu = eps in {1e-2 .. 1e-5} and kappa = eps^2 gamma, HLLC, FV sub-cell
    shock capturing with Persson thresholds -6 / -8, Dirichlet boundaries (the initial states),
    explicit LSRK4 at CFL 0.1, end time 0.11. T = 0.85 (the paper's temperature elsewhere)."""
    return Workload(f"riemann_1d_sharp_E{nelem}_N{N}_eps{eps:g}", 1, (nelem,), N, 0, kappa=eps * eps * gamma,
                    alpha=100.0, beta=1e-3, mu=eps, cfl=0.1, steps=0,
                    extra={"ic": "riemann", "rho_left": 2.0, "rho_right": 0.1, "x0": 0.5, "flux": "hllc",
                           "ind_upper": -6.0, "ind_lower": -8.0, "t_end": 0.11})


def coalescence_2d(alpha=1e2, nelem=128, N=4):
    """2D coalescence of two liquid droplets: 128^2 elements, N=4, radii 0.15 / 0.12 with
    centres 0.3 apart, alpha in {1e2, 1e3, 1e4}, beta=1e-3, mu=2e-3, +-1e-4 noise on rho."""
    return Workload(f"coalescence_2d_E{nelem}x{nelem}_N{N}_alpha{alpha:g}", 2, (nelem, nelem), N, 0,
                    alpha=alpha, mu=2e-3, steps=20000,
                    extra={"ic": "droplets", "centres": ((0.35, 0.5), (0.65, 0.5)), "radii": (0.15, 0.12),
                           "noise": 1e-4, "seed": SEED})


def head_on_collision_3d(we=40.0, nelem=64, N=3):
    """3D head-on droplet collision: 64^3 elements, N=3 (16.8M nodes x 5 variables), radius 0.2,
    centres (0.25,.5,.5) / (0.75,.5,.5), We in {10, 40, 80}, alpha=1e3, beta=1e-3, mu=1e-3."""
    return Workload(f"head_on_collision_3d_E{nelem}^3_N{N}_We{we:g}", 3, (nelem, nelem, nelem), N, 0,
                    steps=5000, extra={"ic": "collision", "we": we, "radius": 0.2})


def serving_batch_3d(n=32, seed=SEED, e_range=(16, 48), n_choices=(3, 4), we_range=(5.0, 100.0),
                     impact_max=0.5, radius=0.2):
    """Batch of n 3D head-on collision instances of uneven size: elements per direction
    uniform in e_range, N uniform in n_choices, We uniform in we_range, impact parameter
    uniform in [0, impact_max] x 2 radius (centres offset in y), seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        ne = int(rng.integers(e_range[0], e_range[1] + 1))
        N = int(rng.choice(n_choices))
        we = float(rng.uniform(*we_range))
        b = float(rng.uniform(0.0, impact_max)) * 2.0 * radius
        c = ((0.25, 0.5 - b / 2, 0.5), (0.75, 0.5 + b / 2, 0.5))
        out.append(Workload(f"collision_{i}_E{ne}^3_N{N}_We{we:.1f}_b{b:.3f}", 3, (ne, ne, ne), N, 0,
                            extra={"ic": "collision", "we": we, "radius": radius, "centres": c}))
    return out
