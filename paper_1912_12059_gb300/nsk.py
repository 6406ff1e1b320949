"""Thin ctypes binding of libnsk.so (include/nsk.h).

Argument marshalling only: every step of the discretisation runs in the CUDA
library. Host arrays are numpy float64 C-contiguous arrays; device arrays are
torch CUDA float64 tensors (contiguous), passed by pointer with where=DEVICE on
the context's stream. If the library is missing the import of this module
still works, but every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "libnsk.so"

NSK_OK = 0
NSK_ERR_ARG = -1
NSK_ERR_CUDA = -2
NSK_ERR_NONPHYSICAL = -3
NSK_ERR_TIMEOUT = -4
NSK_ERR_STATE = -5
NSK_ERR_NOMEM = -6
NSK_ERR_IO = -7
NSK_ERR_BOUNDS = -8
NSK_NODES_GAUSS = 0
NSK_NODES_GAUSS_LOBATTO = 1
NSK_FP64 = 0
NSK_FP32_MIXED = 1
NSK_HOST = 0
NSK_DEVICE = 1
NSK_C_EXPLICIT = 0
NSK_C_LEARNED = 1
NSK_FLUX_LF = 0
NSK_FLUX_HLLC = 1
NSK_MODEL_RELAXATION = 0
NSK_MODEL_NSK = 1

#: every symbol include/nsk.h declares, with (restype, argtypes)
_dp = C.POINTER(C.c_double)
SIGNATURES = {
    "nsk_init_mesh": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), _dp, _dp, C.c_int, C.c_int,
                                C.c_int, C.c_void_p]),
    "nsk_set_params": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
    "nsk_set_c_dissipation": (C.c_int, [C.c_void_p, C.c_int]),
    "nsk_set_flux": (C.c_int, [C.c_void_p, C.c_int]),
    "nsk_set_model": (C.c_int, [C.c_void_p, C.c_int]),
    "nsk_set_subcell": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double]),
    "nsk_set_dirichlet": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp]),
    "nsk_set_subcell_flags": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "nsk_get_subcell": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), _dp]),
    "nsk_subcell_switch": (C.c_int, [C.c_void_p]),
    "nsk_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "nsk_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "nsk_node_coords": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "nsk_rhs": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_int]),
    "nsk_lift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "nsk_compute_dt": (C.c_int, [C.c_void_p, C.c_double, _dp]),
    "nsk_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "nsk_step_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int]),
    "nsk_step_esdirk": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                  C.c_int, C.POINTER(C.c_longlong)]),
    "nsk_diagnostics": (C.c_int, [C.c_void_p, _dp, _dp, _dp]),
    "nsk_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "nsk_launch_count": (C.c_longlong, [C.c_void_p]),
    "nsk_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "nsk_get_profile": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_longlong), C.c_int, C.c_int]),
    "nsk_rhs_static_scratch": (C.c_int, [C.c_int, C.POINTER(C.c_int), _dp, _dp, C.c_int, C.c_int, C.c_double,
                                         C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                         C.c_void_p]),
    "nsk_static_scratch_bytes": (C.c_longlong, []),
    "nsk_set_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "nsk_get_schedule": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "nsk_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp]),
    "nsk_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]),
    "nsk_measure_fma_rate": (C.c_int, [C.c_int, C.c_int, _dp, _dp, C.c_void_p]),
    "nsk_save_checkpoint": (C.c_int, [C.c_void_p, C.c_char_p, C.c_double, C.c_longlong]),
    "nsk_load_checkpoint": (C.c_int, [C.c_void_p, C.c_char_p, _dp, C.POINTER(C.c_longlong)]),
    "nsk_batch_step": (C.c_int, [C.c_void_p, C.c_int, C.c_double, _dp, _dp]),
    "nsk_batch_set_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "nsk_batch_get_schedule": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "nsk_batch_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _dp]),
    "nsk_batch_launch_count": (C.c_longlong, [C.c_void_p]),
    "nsk_batch_uses_graph": (C.c_int, [C.c_void_p]),
    "nsk_batch_set_timeout": (C.c_int, [C.c_void_p, C.c_double]),
    "nsk_test_hook_block_batch_barrier": (C.c_int, [C.c_void_p]),
    "nsk_test_hook_tc_grid_cap": (C.c_int, [C.c_int]),
    "nsk_test_hook_mlp_fwd_kernel": (C.c_int, [C.c_int]),
    "nsk_test_hook_math": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "nsk_test_hook_corrupt_neighbours": (C.c_int, [C.c_void_p]),
    "nsk_batch_destroy": (None, [C.c_void_p]),
    "nsk_gemm_bf16": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nsk_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_void_p]),
    "nsk_mlp_num_params": (C.c_longlong, [C.c_void_p]),
    "nsk_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong]),
    "nsk_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong]),
    "nsk_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "nsk_mlp_set_fused_forward": (C.c_int, [C.c_void_p, C.c_int]),
    "nsk_mlp_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, _dp]),
    "nsk_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, _dp]),
    "nsk_mlp_launch_count": (C.c_longlong, [C.c_void_p]),
    "nsk_mlp_destroy": (None, [C.c_void_p]),
    "nsk_set_closure": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double]),
    "nsk_closure_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), _dp, C.POINTER(C.c_longlong)]),
    "nsk_closure_features": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nsk_closure_targets": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nsk_closure_apply": (C.c_int, [C.c_void_p]),
    "nsk_closure_judge": (C.c_int, [C.c_void_p, _dp]),
    "nsk_error_string": (C.c_char_p, [C.c_int]),
    "nsk_destroy": (None, [C.c_void_p]),
}

_lib = None


class NskError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = error_string(code) if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")


def load_library(path: str | Path | None = None):
    """Load libnsk.so (built by build.build_library()), or the library the environment variable
    NSK_LIBRARY names (e.g. the bounds-checking libnsk_check.so); raises if it is absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else Path(os.environ.get("NSK_LIBRARY") or LIB_PATH)
    if not p.exists():
        raise RuntimeError(f"libnsk.so not found at {p}: build it with paper_1912_12059_gb300.build.build_library() "
                           "(there is no CPU fallback)")
    L = C.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def error_string(code: int) -> str:
    return load_library().nsk_error_string(code).decode()


def _check(code: int, what: str):
    if code != NSK_OK:
        raise NskError(code, what)


def _buf(a, nvals: int, writable: bool):
    """(pointer, where, keepalive) for a numpy host array or a torch CUDA tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != nvals:
            raise ValueError(f"need a C-contiguous float64 array of {nvals} values")
        if writable and not a.flags.writeable:
            raise ValueError("output array is read-only")
        return C.c_void_p(a.ctypes.data), NSK_HOST
    try:
        import torch
    except ImportError as exc:  # pragma: no cover
        raise TypeError("expected a numpy array") from exc
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != nvals:
            raise ValueError(f"need a contiguous float64 tensor of {nvals} values")
        return C.c_void_p(a.data_ptr()), (NSK_DEVICE if a.is_cuda else NSK_HOST)
    raise TypeError("expected a numpy array or a torch tensor")


# ---- same-name wrappers of the C entry points ----

def nsk_init_mesh(dim, nelem, lo, hi, N, node_type=NSK_NODES_GAUSS, precision=NSK_FP64, stream=None):
    L = load_library()
    ctx = C.c_void_p()
    ne = (C.c_int * 3)(*(list(nelem) + [1] * (3 - len(nelem))))
    clo = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    chi = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    _check(L.nsk_init_mesh(C.byref(ctx), dim, ne, clo, chi, N, node_type, precision,
                           C.c_void_p(stream) if stream else None), "nsk_init_mesh")
    return ctx


def nsk_set_params(ctx, T, kappa, alpha, beta, mu):
    _check(load_library().nsk_set_params(ctx, T, kappa, alpha, beta, mu), "nsk_set_params")


def nsk_set_c_dissipation(ctx, on):
    _check(load_library().nsk_set_c_dissipation(ctx, int(bool(on))), "nsk_set_c_dissipation")


def nsk_rhs_static_scratch(dim, nelem, lo, hi, N, node_type, T, kappa, alpha, beta, mu, U, Ut, stream=None):
    """Residual of the device tensor U into the device tensor Ut without any device allocation
    (see include/nsk.h); returns the status code (0 = ok)."""
    ne = (C.c_int * 3)(*(list(nelem) + [1] * (3 - len(nelem))))
    clo = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    chi = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    return load_library().nsk_rhs_static_scratch(dim, ne, clo, chi, N, node_type, T, kappa, alpha, beta, mu,
                                                 C.c_void_p(U.data_ptr()), C.c_void_p(Ut.data_ptr()),
                                                 C.c_void_p(stream) if stream else None)


def _test_hook_tc_grid_cap(max_ctas):
    """Test-only (include/nsk_test_hooks.h): cap the persistent tensor-core grids (0: no cap)."""
    _check(load_library().nsk_test_hook_tc_grid_cap(int(max_ctas)), "nsk_test_hook_tc_grid_cap")


def _test_hook_mlp_fwd_kernel(which):
    """Test-only (include/nsk_test_hooks.h): the fused forward's kernel, 0 the warp-specialised
    TMA kernel where it applies, 1 always the stage-by-stage kernel."""
    _check(load_library().nsk_test_hook_mlp_fwd_kernel(int(which)), "nsk_test_hook_mlp_fwd_kernel")


def _test_hook_math(fn, x, y, stream=None):
    """Test-only (include/nsk_test_hooks.h): the stage kernels' FP64 reciprocal (fn 0) or square
    root (fn 1) of the float64 CUDA tensor x into y."""
    _check(load_library().nsk_test_hook_math(int(fn), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                             int(x.numel()), C.c_void_p(stream) if stream else None),
           "nsk_test_hook_math")


def measure_fma_rate(precision=NSK_FP64, iters=1 << 16, stream=None):
    """Measured FMA throughput of the current device, (TFLOP/s, ms of the timed launch)."""
    tf, ms = C.c_double(), C.c_double()
    _check(load_library().nsk_measure_fma_rate(int(precision), int(iters), C.byref(tf), C.byref(ms),
                                               C.c_void_p(stream) if stream else None), "nsk_measure_fma_rate")
    return tf.value, ms.value


def nsk_destroy(ctx):
    load_library().nsk_destroy(ctx)


class Solver:
    """One context: mesh, parameters and state on the current CUDA device."""

    def __init__(self, dim, nelem, N, lo=None, hi=None, node_type=NSK_NODES_GAUSS, precision=NSK_FP64,
                 stream=None):
        self.dim = dim
        lo = lo if lo is not None else [0.0] * dim
        hi = hi if hi is not None else [1.0] * dim
        self.ctx = nsk_init_mesh(dim, nelem, lo, hi, N, node_type, precision, stream)
        L = load_library()
        E, npe, nv = C.c_longlong(), C.c_int(), C.c_int()
        _check(L.nsk_get_sizes(self.ctx, C.byref(E), C.byref(npe), C.byref(nv)), "nsk_get_sizes")
        self.E, self.npe, self.nvar = E.value, npe.value, nv.value
        self.nq = dim * (dim + 1)
        self.N = N
        self.precision = precision

    # -- lifecycle --
    def close(self):
        if self.ctx:
            nsk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.nvar, self.E, self.npe)

    @property
    def n_nodes(self):
        return self.E * self.npe

    # -- calls --
    def set_params(self, T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3):
        nsk_set_params(self.ctx, T, kappa, alpha, beta, mu)

    def set_c_dissipation(self, on):
        nsk_set_c_dissipation(self.ctx, on)

    def set_flux(self, flux):
        """NSK_FLUX_LF (default) or NSK_FLUX_HLLC."""
        _check(load_library().nsk_set_flux(self.ctx, int(flux)), "nsk_set_flux")

    def set_model(self, model):
        """NSK_MODEL_RELAXATION (default, state rho, m, c) or NSK_MODEL_NSK (original NSK
        equations, state rho, m); a new set_state is required afterwards."""
        L = load_library()
        _check(L.nsk_set_model(self.ctx, int(model)), "nsk_set_model")
        E, npe, nv = C.c_longlong(), C.c_int(), C.c_int()
        _check(L.nsk_get_sizes(self.ctx, C.byref(E), C.byref(npe), C.byref(nv)), "nsk_get_sizes")
        self.nvar = nv.value

    def set_subcell(self, on=True, ind_upper=-6.0, ind_lower=-8.0):
        """Finite-volume sub-cell shock capturing with the Persson indicator (1D, FP64, model II)."""
        _check(load_library().nsk_set_subcell(self.ctx, int(bool(on)), float(ind_upper), float(ind_lower)),
               "nsk_set_subcell")

    def set_dirichlet(self, Ub_lo=None, Ub_hi=None):
        """Dirichlet boundary states (rho, m, c) outside x = lo and x = hi (1D); None: periodic."""
        on = Ub_lo is not None
        lo = (C.c_double * 3)(*(Ub_lo if on else (0.0, 0.0, 0.0)))
        hi = (C.c_double * 3)(*(Ub_hi if on else (0.0, 0.0, 0.0)))
        _check(load_library().nsk_set_dirichlet(self.ctx, int(on), lo, hi), "nsk_set_dirichlet")

    def set_subcell_flags(self, flags):
        fl = np.ascontiguousarray(flags, dtype=np.int32)
        assert fl.size == self.E
        _check(load_library().nsk_set_subcell_flags(self.ctx, fl.ctypes.data_as(C.POINTER(C.c_int))),
               "nsk_set_subcell_flags")

    def subcell(self):
        """(flags, indicator of the last switch pass), host arrays of E."""
        fl = np.zeros(self.E, dtype=np.int32)
        ind = np.zeros(self.E)
        _check(load_library().nsk_get_subcell(self.ctx, fl.ctypes.data_as(C.POINTER(C.c_int)),
                                              ind.ctypes.data_as(C.POINTER(C.c_double))), "nsk_get_subcell")
        return fl, ind

    def subcell_switch(self):
        _check(load_library().nsk_subcell_switch(self.ctx), "nsk_subcell_switch")

    def set_state(self, U):
        ptr, where = _buf(U, self.nvar * self.n_nodes, False)
        _check(load_library().nsk_set_state(self.ctx, ptr, where), "nsk_set_state")

    def get_state(self, out=None):
        out = np.empty(self.shape) if out is None else out
        ptr, where = _buf(out, self.nvar * self.n_nodes, True)
        _check(load_library().nsk_get_state(self.ctx, ptr, where), "nsk_get_state")
        return out

    def node_coords(self, out=None):
        out = np.empty((self.dim, self.E, self.npe)) if out is None else out
        ptr, where = _buf(out, self.dim * self.n_nodes, True)
        _check(load_library().nsk_node_coords(self.ctx, ptr, where), "nsk_node_coords")
        return out

    def rhs(self, t=0.0, out=None):
        out = np.empty(self.shape) if out is None else out
        ptr, where = _buf(out, self.nvar * self.n_nodes, True)
        _check(load_library().nsk_rhs(self.ctx, t, ptr, where), "nsk_rhs")
        return out

    def lift(self, out=None):
        out = np.empty((self.nq, self.E, self.npe)) if out is None else out
        ptr, where = _buf(out, self.nq * self.n_nodes, True)
        _check(load_library().nsk_lift(self.ctx, ptr, where), "nsk_lift")
        return out

    def compute_dt(self, cfl):
        dt = C.c_double()
        _check(load_library().nsk_compute_dt(self.ctx, cfl, C.byref(dt)), "nsk_compute_dt")
        return dt.value

    def step(self, dt, nsteps=1):
        _check(load_library().nsk_step(self.ctx, dt, nsteps), "nsk_step")

    def step_host(self, U_in, dt, nsteps=1, out=None):
        """nsk_step_host: the state from host memory (U_in: a float64 numpy array or CPU tensor,
        pinned for the full copy rate), nsteps steps, the final state into out (default U_in)."""
        out = U_in if out is None else out
        pin, w_in = _buf(U_in, self.nvar * self.n_nodes, False)
        pout, w_out = _buf(out, self.nvar * self.n_nodes, True)
        if w_in != NSK_HOST or w_out != NSK_HOST:
            raise ValueError("step_host takes host arrays")
        _check(load_library().nsk_step_host(self.ctx, pin, pout, dt, nsteps), "nsk_step_host")
        return out

    def step_esdirk(self, dt, nsteps=1, newton_tol=1e-10, krylov_tol=1e-3, krylov_dim=30, max_krylov=600,
                    block_precond=False):
        """Implicit six-stage ESDIRK4 steps (Jacobian-free Newton-Krylov, optionally with the
        element-block preconditioner); returns the statistics {newton, krylov, rhs, failed}
        summed over the call."""
        st = (C.c_longlong * 4)()
        _check(load_library().nsk_step_esdirk(self.ctx, float(dt), int(nsteps), float(newton_tol), float(krylov_tol),
                                              int(krylov_dim), int(max_krylov), int(bool(block_precond)), st),
               "nsk_step_esdirk")
        return {"newton": st[0], "krylov": st[1], "rhs": st[2], "failed": st[3]}

    def save_checkpoint(self, path, t=0.0, step=0):
        """Write the state (FP64), the parameters and the caller's time and step counter to path
        (the binary format of nsk_save_checkpoint in include/nsk.h)."""
        _check(load_library().nsk_save_checkpoint(self.ctx, str(path).encode(), float(t), int(step)),
               "nsk_save_checkpoint")

    def load_checkpoint(self, path):
        """Read a checkpoint of a context with this mesh; sets the parameters and the state and
        returns (t, step). Stepping on gives the same bits as never stopping."""
        t, step = C.c_double(), C.c_longlong()
        _check(load_library().nsk_load_checkpoint(self.ctx, str(path).encode(), C.byref(t), C.byref(step)),
               "nsk_load_checkpoint")
        return t.value, step.value

    def diagnostics(self):
        m, e, l2 = C.c_double(), C.c_double(), C.c_double()
        _check(load_library().nsk_diagnostics(self.ctx, C.byref(m), C.byref(e), C.byref(l2)), "nsk_diagnostics")
        return m.value, e.value, l2.value

    def set_schedule(self, tpb=256, fused_face=0):
        """fused_face: 0 separate face pass, 1 (or True) face fluxes in the volume kernel, 2 the
        lean two-launch stage (lifting recomputed on chip by the volume kernel), 3 the
        single-block schedule for small meshes (a whole call in one launch), 4 the separate face
        pass with line-per-thread lifting and volume kernels (FP32, 3D, N = 3)."""
        _check(load_library().nsk_set_schedule(self.ctx, tpb, int(fused_face)), "nsk_set_schedule")

    def get_schedule(self):
        """(tpb, fused_face) with fused_face 0 to 4 (see set_schedule)."""
        t, f = C.c_int(), C.c_int()
        _check(load_library().nsk_get_schedule(self.ctx, C.byref(t), C.byref(f)), "nsk_get_schedule")
        return t.value, f.value

    def autotune(self):
        """Time the stage schedules on the current state; keep and return the fastest
        (tpb, fused_face, ms)."""
        t, f, ms = C.c_int(), C.c_int(), C.c_double()
        _check(load_library().nsk_autotune(self.ctx, C.byref(t), C.byref(f), C.byref(ms)), "nsk_autotune")
        return t.value, f.value, ms.value

    # -- learned c-closure --
    @property
    def closure_inputs(self):
        """Network inputs of the closure: hi and lo BF16 parts of npe + 2 dim features."""
        return 2 * (self.npe + 2 * self.dim)

    def set_closure(self, mlp=None, judge_every=10, eta_max=0.5):
        """mlp=None switches back to the explicit c equation."""
        mode = NSK_C_LEARNED if mlp is not None else NSK_C_EXPLICIT
        _check(load_library().nsk_set_closure(self.ctx, mode, mlp.h if mlp is not None else None, judge_every,
                                              eta_max), "nsk_set_closure")
        self._mlp = mlp

    def closure_status(self):
        m, e, f = C.c_int(), C.c_double(), C.c_longlong()
        _check(load_library().nsk_closure_status(self.ctx, C.byref(m), C.byref(e), C.byref(f)), "nsk_closure_status")
        return {"mode": m.value, "eta": e.value, "fallbacks": f.value}

    def closure_features(self, X):
        """X: torch bfloat16 CUDA tensor [E, n_in_pad]."""
        _check(load_library().nsk_closure_features(self.ctx, C.c_void_p(X.data_ptr())), "nsk_closure_features")

    def closure_targets(self, Y):
        """Y: torch float32 CUDA tensor [E, npe]: (c - rho) / ((kappa/alpha)(2/h)^2)."""
        _check(load_library().nsk_closure_targets(self.ctx, C.c_void_p(Y.data_ptr())), "nsk_closure_targets")

    def closure_apply(self):
        _check(load_library().nsk_closure_apply(self.ctx), "nsk_closure_apply")

    def closure_judge(self):
        e = C.c_double()
        _check(load_library().nsk_closure_judge(self.ctx, C.byref(e)), "nsk_closure_judge")
        return e.value

    KERNELS = ("k_prolong", "k_lift", "k_face", "k_volume", "k_block")

    def set_profiling(self, on=True):
        _check(load_library().nsk_set_profiling(self.ctx, int(bool(on))), "nsk_set_profiling")

    def get_profile(self, reset=False):
        """{kernel: (total ms, launches)} accumulated while profiling was on."""
        nk = len(self.KERNELS)
        ms = (C.c_double * nk)()
        cnt = (C.c_longlong * nk)()
        n = load_library().nsk_get_profile(self.ctx, ms, cnt, nk, int(bool(reset)))
        if n < 0:
            raise NskError(n, "nsk_get_profile")
        return {self.KERNELS[k]: (ms[k], cnt[k]) for k in range(min(n, nk)) if cnt[k] or k < 4}

    @property
    def launch_count(self):
        return int(load_library().nsk_launch_count(self.ctx))


class Batch:
    """Many 3D contexts (N = 3 or 4, same precision) advanced together by one
    persistent launch per RK stage, replayed from a CUDA graph."""

    def __init__(self, solvers):
        self.solvers = list(solvers)  # keep the contexts alive
        self.n = len(self.solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        h = C.c_void_p()
        _check(load_library().nsk_batch_create(C.byref(h), len(self.solvers), arr), "nsk_batch_create")
        self.h = h

    def step(self, nsteps=1, cfl=0.0, timings=False, latencies=False):
        """Advance all instances; cfl > 0 recomputes each instance's dt every step.
        With timings=True returns the per-step wall times in ms; with latencies=True (also)
        the per-instance step latencies, an array [nsteps][instances] in ms (time from the
        step's start until that instance's new state is complete)."""
        ms = (C.c_double * max(nsteps, 1))() if timings else None
        lat = (C.c_double * max(nsteps * self.n, 1))() if latencies else None
        _check(load_library().nsk_batch_step(self.h, nsteps, cfl, ms, lat), "nsk_batch_step")
        out_ms = list(ms)[:nsteps] if timings else None
        if not latencies:
            return out_ms
        L = np.frombuffer(lat, dtype=np.float64, count=nsteps * self.n).reshape(nsteps, self.n).copy()
        return (out_ms, L) if timings else L

    #: values of the `persistent` schedule argument
    PHASES, PERSISTENT, INSTANCES = 0, 1, 2

    def set_schedule(self, tpb=256, fused_face=False, persistent=1):
        """persistent: 1 cooperative persistent kernel, 0 one launch per phase, 2 each instance's
        own stage launches (True/False map to 1/0); fused_face 0 or 1, or with the instance
        schedule also 2 (the lean stage), 4 (the line kernels where they apply) or 5 (each
        instance's own schedule; tpb is then ignored)."""
        _check(load_library().nsk_batch_set_schedule(self.h, tpb, int(fused_face), int(persistent)),
               "nsk_batch_set_schedule")

    def get_schedule(self):
        t, f, p = C.c_int(), C.c_int(), C.c_int()
        _check(load_library().nsk_batch_get_schedule(self.h, C.byref(t), C.byref(f), C.byref(p)),
               "nsk_batch_get_schedule")
        return t.value, f.value, p.value

    def autotune(self):
        """Time all ten schedules on the batch; keep and return (tpb, fused, persistent, ms)."""
        t, f, p, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(load_library().nsk_batch_autotune(self.h, C.byref(t), C.byref(f), C.byref(p), C.byref(ms)),
               "nsk_batch_autotune")
        return t.value, bool(f.value), p.value, ms.value

    def set_timeout(self, seconds):
        _check(load_library().nsk_batch_set_timeout(self.h, seconds), "nsk_batch_set_timeout")

    def _test_hook_block_barrier(self):
        """Test-only (include/nsk_test_hooks.h): make the next grid barrier unreachable."""
        _check(load_library().nsk_test_hook_block_batch_barrier(self.h), "nsk_test_hook_block_batch_barrier")

    @property
    def uses_graph(self):
        return bool(load_library().nsk_batch_uses_graph(self.h))

    @property
    def launch_count(self):
        return int(load_library().nsk_batch_launch_count(self.h))

    def close(self):
        if self.h:
            load_library().nsk_batch_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def _ptr_or_null(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def gemm_bf16(A, B, epilogue=0, bias=None, out=None, hout=None, hout_t=None, zin=None, bias_grad=None, k_split=0,
              err=None, stream=None):
    """C = A . B^T on the tensor cores for torch CUDA tensors (A [M,K], B [N,K] bfloat16, row-major);
    see nsk_gemm_bf16 in include/nsk.h for the epilogues. Returns the status code."""
    M, K = A.shape
    N = B.shape[0]
    lib = load_library()
    return lib.nsk_gemm_bf16(_ptr_or_null(A), _ptr_or_null(B), M, N, K, A.stride(0), B.stride(0), k_split, epilogue,
                             _ptr_or_null(bias), _ptr_or_null(out), out.stride(0) if out is not None else 0,
                             _ptr_or_null(hout), hout.stride(0) if hout is not None else 0, _ptr_or_null(hout_t),
                             hout_t.stride(0) if hout_t is not None else 0, _ptr_or_null(zin),
                             zin.stride(0) if zin is not None else 0, _ptr_or_null(bias_grad), _ptr_or_null(err),
                             C.c_void_p(stream) if stream else None)


class MLP:
    """Per-element network of the learned closure (include/nsk.h: nsk_mlp_*), n_in -> h1 -> h2 -> n_out."""

    def __init__(self, n_in, h1=256, h2=256, n_out=64, max_batch=8192, max_rows=1, stream=None):
        h = C.c_void_p()
        _check(load_library().nsk_mlp_create(C.byref(h), n_in, h1, h2, n_out, max_batch, max_rows,
                                             C.c_void_p(stream) if stream else None), "nsk_mlp_create")
        self.h = h
        self.n_in, self.h1, self.h2, self.n_out = n_in, h1, h2, n_out
        self.max_batch, self.max_rows = max_batch, max_rows
        self.n_in_pad = (n_in + 15) // 16 * 16
        self.n_params = int(load_library().nsk_mlp_num_params(h))

    def layout(self):
        """[(name, shape)] of the flat FP32 parameter vector."""
        return [("W1", (self.h1, self.n_in_pad)), ("b1", (self.h1,)), ("W2", (self.h2, self.h1)), ("b2", (self.h2,)),
                ("W3", (self.n_out, self.h2)), ("b3", (self.n_out,))]

    def unflatten(self, flat):
        out, o = {}, 0
        for name, shape in self.layout():
            n = int(np.prod(shape))
            out[name] = np.asarray(flat[o:o + n]).reshape(shape)
            o += n
        return out

    def init_params(self, seed=0):
        """He-uniform weights, zero biases (seeded)."""
        rng = np.random.Generator(np.random.PCG64(seed))
        parts = []
        for name, shape in self.layout():
            if name.startswith("W"):
                fan_in = self.n_in if name == "W1" else shape[1]
                w = rng.uniform(-1, 1, size=shape) * np.sqrt(6.0 / fan_in)
                if name == "W1":
                    w[:, self.n_in:] = 0.0
                parts.append(w.ravel())
            else:
                parts.append(np.zeros(shape).ravel())
        self.set_params(np.concatenate(parts).astype(np.float32))

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        _check(load_library().nsk_mlp_set_params(self.h, C.c_void_p(flat.ctypes.data), flat.size),
               "nsk_mlp_set_params")

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(load_library().nsk_mlp_get_params(self.h, C.c_void_p(out.ctypes.data), out.size), "nsk_mlp_get_params")
        return out

    def forward(self, X, Y):
        _check(load_library().nsk_mlp_forward(self.h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr())),
               "nsk_mlp_forward")

    def set_fused_forward(self, on):
        """False forces the three-GEMM forward (default: one fused kernel where the network fits)."""
        _check(load_library().nsk_mlp_set_fused_forward(self.h, int(bool(on))), "nsk_mlp_set_fused_forward")

    def gradients(self, X, T):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_double()
        _check(load_library().nsk_mlp_gradients(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                                X.shape[0], C.c_void_p(g.ctypes.data), C.byref(loss)),
               "nsk_mlp_gradients")
        return g, loss.value

    def train_step(self, X, T, lr, want_loss=False):
        loss = C.c_double()
        _check(load_library().nsk_mlp_train_step(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                                 X.shape[0], lr, C.byref(loss) if want_loss else None),
               "nsk_mlp_train_step")
        return loss.value if want_loss else None

    @property
    def launch_count(self):
        return int(load_library().nsk_mlp_launch_count(self.h))

    def close(self):
        if self.h:
            load_library().nsk_mlp_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
