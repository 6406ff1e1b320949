"""TEST INFRASTRUCTURE ONLY: loader of the plain FP64 CPU oracle (nsk_oracle.c).

The oracle restates the discretisation of arXiv:1912.12059 (relaxation model II,
weak-form DGSEM with BR1 lifting, local Lax-Friedrichs flux, five-stage
low-storage RK4) in slow, obviously correct C. Only tests/, the package smoke
check and bench.py's CPU-baseline leg may import this module; the product path
never does. Every function cites the passage of the paper it follows in the C
source.
"""
from __future__ import annotations

import ctypes as C
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "nsk_oracle.c"
HDR = HERE / "nsk_oracle.h"
LIB = HERE / "libnsk_oracle.so"

NODES_GAUSS = 0
NODES_LOBATTO = 1
FLUX_LF = 0    # local Lax-Friedrichs
FLUX_HLLC = 1  # HLLC (barotropic, modified pressure)
MODEL_RELAXATION = 0  # relaxation model II: state (rho, m, c)
MODEL_NSK = 1         # original NSK equations: state (rho, m)


class OrcSetup(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("nelem", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("N", C.c_int),
        ("node_type", C.c_int),
        ("T", C.c_double),
        ("kappa", C.c_double),
        ("alpha", C.c_double),
        ("beta", C.c_double),
        ("mu", C.c_double),
        ("c_dissipation", C.c_int),
        ("flux", C.c_int),
        ("model", C.c_int),
    ]


class OrcFvSetup(C.Structure):
    _fields_ = [
        ("dirichlet", C.c_int),
        ("Ub_lo", C.c_double * 3),
        ("Ub_hi", C.c_double * 3),
        ("ind_upper", C.c_double),
        ("ind_lower", C.c_double),
    ]


LIB_OMP = HERE / "libnsk_oracle_omp.so"


def build_oracle(force: bool = False, parallel: bool = False) -> Path:
    """Compile the oracle with gcc (FP contraction off, so no fused multiply-adds). parallel=True
    builds the same source a second time with OpenMP (-fopenmp) for the timed CPU baseline on all
    host cores: its loops over elements and faces share out iterations that write disjoint
    results, and every sum keeps its order, so both libraries compute the same bits."""
    target = LIB_OMP if parallel else LIB
    if not force and target.exists() and target.stat().st_mtime >= max(SRC.stat().st_mtime, HDR.stat().st_mtime):
        return target
    tmp = target.with_suffix(".so.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(SRC), "-o", str(tmp), "-lm"]
    if parallel:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    tmp.replace(target)
    return target


_libs = {}


def lib(parallel: bool = False):
    """The loaded oracle library: the plain build, or (parallel=True) the OpenMP build."""
    if parallel not in _libs:
        L = C.CDLL(str(build_oracle(parallel=parallel)))
        dp = C.POINTER(C.c_double)
        sp = C.POINTER(OrcSetup)
        for name in ("orc_pressure", "orc_dpressure", "orc_free_energy", "orc_chem_potential"):
            f = getattr(L, name)
            f.restype = C.c_double
            f.argtypes = [C.c_double, C.c_double]
        L.orc_maxwell.argtypes = [C.c_double, dp, dp, dp]
        L.orc_spinodal.argtypes = [C.c_double, dp, dp, dp]
        L.orc_young_laplace.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_nodes.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_lagrange_tables.argtypes = [C.c_int, dp, dp, dp, dp]
        L.orc_lagrange_tables.restype = None
        L.orc_lagrange_eval.argtypes = [C.c_int, dp, C.c_int, C.c_double]
        L.orc_lagrange_eval.restype = C.c_double
        L.orc_lsrk4_coeffs.argtypes = [dp, dp, dp]
        L.orc_lsrk4_coeffs.restype = None
        L.orc_lift.argtypes = [sp, dp, dp]
        L.orc_rhs.argtypes = [sp, dp, dp]
        L.orc_numflux.argtypes = [sp, C.c_int, dp, dp, dp]
        L.orc_lift2.argtypes = [sp, dp, dp]
        L.orc_lsrk4.argtypes = [sp, dp, C.c_double, C.c_int]
        L.orc_timestep.argtypes = [sp, dp, C.c_double, dp]
        L.orc_diagnostics.argtypes = [sp, dp, dp, dp, dp]
        fp = C.POINTER(OrcFvSetup)
        ip = C.POINTER(C.c_int)
        L.orc_fv_tables.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_persson.argtypes = [C.c_int, C.c_int, dp]
        L.orc_persson.restype = C.c_double
        L.orc_fv_rhs.argtypes = [sp, fp, ip, dp, dp]
        L.orc_fv_switch.argtypes = [sp, fp, ip, dp, dp]
        L.orc_fv_lsrk4.argtypes = [sp, fp, ip, dp, C.c_double, C.c_int]
        L.orc_threads.argtypes = []
        _libs[parallel] = L
    return _libs[parallel]


def threads(parallel: bool = False) -> int:
    """Threads the oracle's loops run on in that build (1 for the plain build)."""
    return lib(parallel).orc_threads()


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(f"{what} failed with code {code}")


# ---- thermodynamics ----
def pressure(T, rho):
    return lib().orc_pressure(T, rho)


def dpressure(T, rho):
    return lib().orc_dpressure(T, rho)


def free_energy(T, rho):
    return lib().orc_free_energy(T, rho)


def chem_potential(T, rho):
    return lib().orc_chem_potential(T, rho)


def maxwell(T=0.85):
    v, l, p = C.c_double(), C.c_double(), C.c_double()
    _check(lib().orc_maxwell(T, C.byref(v), C.byref(l), C.byref(p)), "orc_maxwell")
    return v.value, l.value, p.value


def spinodal(T=0.85):
    a, b, s = C.c_double(), C.c_double(), C.c_double()
    _check(lib().orc_spinodal(T, C.byref(a), C.byref(b), C.byref(s)), "orc_spinodal")
    return a.value, b.value, s.value


def young_laplace(T, sigma, r):
    l, v = C.c_double(), C.c_double()
    _check(lib().orc_young_laplace(T, sigma, r, C.byref(l), C.byref(v)), "orc_young_laplace")
    return l.value, v.value


# ---- basis ----
def nodes(N, node_type=NODES_GAUSS):
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    _check(lib().orc_nodes(N, node_type, _ptr(xi), _ptr(w)), "orc_nodes")
    return xi, w


def lagrange_tables(N, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    D = np.zeros((N + 1) * (N + 1))
    Lm = np.zeros(N + 1)
    Lp = np.zeros(N + 1)
    lib().orc_lagrange_tables(N, _ptr(xi), _ptr(D), _ptr(Lm), _ptr(Lp))
    return D.reshape(N + 1, N + 1), Lm, Lp


def lsrk4_coeffs():
    A, B, Cc = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().orc_lsrk4_coeffs(_ptr(A), _ptr(B), _ptr(Cc))
    return A, B, Cc


def fv_tables(N, node_type=NODES_GAUSS):
    """Sub-cell mean matrix M[j][i] (mean of l_i over sub-cell j of N+1) and its inverse."""
    M = np.zeros((N + 1) * (N + 1))
    Minv = np.zeros((N + 1) * (N + 1))
    _check(lib().orc_fv_tables(N, node_type, _ptr(M), _ptr(Minv)), "orc_fv_tables")
    return M.reshape(N + 1, N + 1), Minv.reshape(N + 1, N + 1)


def persson(u, node_type=NODES_GAUSS):
    """Persson-Peraire indicator of the nodal values u (N + 1 of them)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_persson(len(u) - 1, node_type, _ptr(u))


# ---- discretisation ----
class Oracle:
    """One mesh + parameter set of the oracle; arrays in the canonical layout
    [nvar][E][npe] (variables rho, rho v_1..rho v_dim, c)."""

    def __init__(self, dim, nelem, lo, hi, N, node_type=NODES_GAUSS, T=0.85, kappa=1e-4, alpha=1e3,
                 beta=1e-3, mu=1e-3, c_dissipation=0, flux=FLUX_LF, model=MODEL_RELAXATION, parallel=False):
        self.L = lib(parallel)  # the plain build, or the OpenMP build of the same source
        s = OrcSetup()
        s.dim = dim
        ne = list(nelem) + [1] * (3 - len(nelem))
        lo = list(lo) + [0.0] * (3 - len(lo))
        hi = list(hi) + [1.0] * (3 - len(hi))
        for k in range(3):
            s.nelem[k] = ne[k] if k < dim else 1
            s.lo[k] = lo[k]
            s.hi[k] = hi[k]
        s.N = N
        s.node_type = node_type
        s.T, s.kappa, s.alpha, s.beta, s.mu = T, kappa, alpha, beta, mu
        s.c_dissipation = c_dissipation
        s.flux = flux
        s.model = model
        self.s = s
        self.dim = dim
        self.N = N
        self.np = N + 1
        self.npe = (N + 1) ** dim
        self.E = int(np.prod(ne[:dim]))
        self.nvar = dim + 1 if model == MODEL_NSK else dim + 2
        self.nq = dim * (dim + 1)
        self.nelem = ne[:dim]
        self.lo, self.hi = lo[:dim], hi[:dim]
        self.xi, self.w = nodes(N, node_type)

    @property
    def shape(self):
        return (self.nvar, self.E, self.npe)

    def coords(self):
        """Physical node coordinates [dim][E][npe] of the affine element maps:
        x_k = lo_k + h_k (e_k + (xi_{i_k} + 1)/2) with e_k the element's and i_k the node's index
        along direction k (lexicographic, x fastest)."""
        x = np.zeros((self.dim, self.E, self.npe))
        h = [(self.hi[k] - self.lo[k]) / self.nelem[k] for k in range(self.dim)]
        e = np.arange(self.E)
        n = np.arange(self.npe)
        se, sn = 1, 1
        for k in range(self.dim):
            ec = (e // se) % self.nelem[k]
            i = (n // sn) % self.np
            x[k] = self.lo[k] + h[k] * (ec[:, None] + 0.5 * (self.xi[i][None, :] + 1.0))
            se *= self.nelem[k]
            sn *= self.np
        return x

    def lift(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        Q = np.zeros((self.nq, self.E, self.npe))
        _check(self.L.orc_lift(C.byref(self.s), _ptr(U), _ptr(Q)), "orc_lift")
        return Q

    def rhs(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        R = np.zeros_like(U)
        _check(self.L.orc_rhs(C.byref(self.s), _ptr(U), _ptr(R)), "orc_rhs")
        return R

    def lift2(self, U):
        """Original NSK: the second lifting, lap rho = div(grad rho), [E][npe]."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        Q2 = np.zeros((self.E, self.npe))
        _check(self.L.orc_lift2(C.byref(self.s), _ptr(U), _ptr(Q2)), "orc_lift2")
        return Q2

    def numflux(self, k, UL, UR):
        """Convective numerical flux (LF or HLLC per the setup) of one face with normal +e_k."""
        UL = np.ascontiguousarray(UL, dtype=np.float64)
        UR = np.ascontiguousarray(UR, dtype=np.float64)
        F = np.zeros(self.nvar)
        _check(self.L.orc_numflux(C.byref(self.s), k, _ptr(UL), _ptr(UR), _ptr(F)), "orc_numflux")
        return F

    def step(self, U, dt, nsteps):
        U = np.array(U, dtype=np.float64, order="C", copy=True)
        _check(self.L.orc_lsrk4(C.byref(self.s), _ptr(U), dt, nsteps), "orc_lsrk4")
        return U

    def timestep(self, U, cfl):
        U = np.ascontiguousarray(U, dtype=np.float64)
        dt = C.c_double()
        _check(self.L.orc_timestep(C.byref(self.s), _ptr(U), cfl, C.byref(dt)), "orc_timestep")
        return dt.value

    def diagnostics(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        m, e, l2 = C.c_double(), C.c_double(), C.c_double()
        _check(self.L.orc_diagnostics(C.byref(self.s), _ptr(U), C.byref(m), C.byref(e), C.byref(l2)),
               "orc_diagnostics")
        return m.value, e.value, l2.value

    # ---- sub-cell shock capturing and Dirichlet boundaries (dim = 1, model II) ----
    def fv_setup(self, dirichlet=False, Ub_lo=(1.0, 0.0, 1.0), Ub_hi=(1.0, 0.0, 1.0), ind_upper=-6.0,
                 ind_lower=-8.0):
        f = OrcFvSetup()
        f.dirichlet = 1 if dirichlet else 0
        for v in range(3):
            f.Ub_lo[v] = Ub_lo[v]
            f.Ub_hi[v] = Ub_hi[v]
        f.ind_upper, f.ind_lower = ind_upper, ind_lower
        self.f = f
        return f

    def fv_rhs(self, U, flags):
        U = np.ascontiguousarray(U, dtype=np.float64)
        fl = np.ascontiguousarray(flags, dtype=np.int32)
        R = np.zeros_like(U)
        _check(self.L.orc_fv_rhs(C.byref(self.s), C.byref(self.f), fl.ctypes.data_as(C.POINTER(C.c_int)), _ptr(U),
                                _ptr(R)), "orc_fv_rhs")
        return R

    def fv_switch(self, U, flags):
        """Indicator of every element and the switches it triggers: (U', flags', ind)."""
        U = np.array(U, dtype=np.float64, order="C", copy=True)
        fl = np.array(flags, dtype=np.int32, order="C", copy=True)
        ind = np.zeros(self.E)
        _check(self.L.orc_fv_switch(C.byref(self.s), C.byref(self.f), fl.ctypes.data_as(C.POINTER(C.c_int)), _ptr(U),
                                   _ptr(ind)), "orc_fv_switch")
        return U, fl, ind

    def fv_step(self, U, flags, dt, nsteps):
        U = np.array(U, dtype=np.float64, order="C", copy=True)
        fl = np.array(flags, dtype=np.int32, order="C", copy=True)
        _check(self.L.orc_fv_lsrk4(C.byref(self.s), C.byref(self.f), fl.ctypes.data_as(C.POINTER(C.c_int)), _ptr(U),
                                  dt, nsteps), "orc_fv_lsrk4")
        return U, fl
