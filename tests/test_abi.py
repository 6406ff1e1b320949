"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no GPU: only calls that fail argument validation before touching CUDA)."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    """Every nsk_* function declared in include/*.h (the boundary nsk.h and the test hooks)."""
    names = set()
    for h in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(nsk_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("nsk_init_mesh", "nsk_set_params", "nsk_set_state", "nsk_rhs", "nsk_step", "nsk_get_state"):
        assert required in names


def test_library_exports_every_declared_symbol(nsk_lib):
    from paper_1912_12059_gb300 import nsk

    for name in _declared():
        assert hasattr(nsk_lib, name), name
        assert name in nsk.SIGNATURES, f"binding lacks {name}"
    out = subprocess.run(["nm", "-D", "--defined-only", str(nsk.LIB_PATH)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(nsk_[a-z0-9_]+)\b", out))
    assert set(_declared()) <= exported
    assert not re.search(r"\borc_", out), "product library must not contain oracle code"


def test_error_strings_and_argument_validation(nsk_lib):
    from paper_1912_12059_gb300 import nsk

    assert nsk.error_string(nsk.NSK_ERR_NONPHYSICAL).startswith("non-physical")
    assert nsk.error_string(12345) == "unknown error"
    ctx = C.c_void_p()
    ne = (C.c_int * 3)(4, 4, 4)
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    # invalid dimension, degree, node type and precision are rejected before any CUDA call
    assert nsk_lib.nsk_init_mesh(C.byref(ctx), 4, ne, lo, hi, 3, 0, 0, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_init_mesh(C.byref(ctx), 3, ne, lo, hi, 9, 0, 0, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_init_mesh(C.byref(ctx), 3, ne, lo, hi, 3, 7, 0, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_init_mesh(C.byref(ctx), 3, ne, lo, hi, 3, 0, 5, None) == nsk.NSK_ERR_ARG
    bad_hi = (C.c_double * 3)(0, 1, 1)
    assert nsk_lib.nsk_init_mesh(C.byref(ctx), 3, ne, lo, bad_hi, 3, 0, 0, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_set_params(None, 0.85, 1e-4, 1e3, 1e-3, 1e-3) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_launch_count(None) == -1
    # the sub-cell, boundary and implicit entries validate their context first
    ub = (C.c_double * 3)(1.0, 0.0, 1.0)
    assert nsk_lib.nsk_set_subcell(None, 1, -6.0, -8.0) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_set_dirichlet(None, 1, ub, ub) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_set_subcell_flags(None, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_get_subcell(None, None, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_subcell_switch(None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_step_esdirk(None, 1e-5, 1, 1e-10, 1e-3, 30, 600, 0, None) == nsk.NSK_ERR_ARG
    # the host-state step validates its context, buffers, step and count before any copy
    buf = (C.c_double * 4)()
    assert nsk_lib.nsk_step_host(None, buf, buf, 1e-5, 1) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_step_host(None, None, buf, 1e-5, 1) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_step_host(None, buf, buf, float("nan"), 1) == nsk.NSK_ERR_ARG
    # the closure and batch calls in the forms the boundary documents (readings R30, R31)
    assert nsk_lib.nsk_set_closure(None, nsk.NSK_C_LEARNED, None, 10, 0.5) == nsk.NSK_ERR_ARG
    lat = (C.c_double * 4)()
    assert nsk_lib.nsk_batch_step(None, 1, 0.0, None, lat) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_set_schedule(None, 256, 2) == nsk.NSK_ERR_ARG
    # measurement and test hooks validate before touching CUDA
    assert nsk_lib.nsk_measure_fma_rate(7, 100, None, None, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_measure_fma_rate(nsk.NSK_FP64, 0, None, None, None) == nsk.NSK_ERR_ARG
    assert nsk_lib.nsk_test_hook_tc_grid_cap(-1) == nsk.NSK_ERR_ARG
    nsk_lib.nsk_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1912_12059_gb300 import nsk

    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nsk.load_library(tmp_path / "absent.so")


def test_product_never_imports_the_oracle():
    pkg = ROOT / "paper_1912_12059_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")) + list(pkg.rglob("*.h")):
        text = f.read_text()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
        assert "nsk_oracle" not in text, f
