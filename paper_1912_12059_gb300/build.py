"""Build libnsk.so (the CUDA library behind include/nsk.h) in-tree for sm_103a.

Each .cu translation unit compiles in parallel with nvcc; the objects are
linked into paper_1912_12059_gb300/libnsk.so. A rebuild happens only when a
source or header is newer than the library.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "libnsk.so"
# the bounds-checking build (-DNSK_BOUNDS_CHECK): every neighbour index checked, failures reported
# as NSK_ERR_BOUNDS instead of faulting; a debugging aid, built on request only
BUILD_CHECK = PKG / "_build_check"
LIB_CHECK = PKG / "libnsk_check.so"

SOURCES = ["nsk_api.cu", "nsk_aux.cu", "nsk_dg1.cu", "nsk_dg2.cu", "nsk_dg3.cu", "nsk_dg3f.cu", "nsk_batch.cu",
           "nsk_mlp.cu", "nsk_orig.cu", "nsk_fv.cu", "nsk_implicit.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (Path(cand).exists() or cand == "nvcc"):
            return cand
    return "nvcc"


def _stale(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh"))
    deps += list(INCLUDE.glob("*.h")) + [Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps if d.exists())


def build_library(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> Path:
    """Compile every CUDA source for sm_103a and link libnsk.so (or, bounds_check=True, the
    bounds-checking libnsk_check.so); return its path."""
    lib, build = (LIB_CHECK, BUILD_CHECK) if bounds_check else (LIB, BUILD)
    if not force and not _stale(lib):
        return lib
    build.mkdir(exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    extra = ["-DNSK_BOUNDS_CHECK"] if bounds_check else []
    for src in SOURCES:
        obj = build / (Path(src).stem + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", str(INCLUDE), "-I", str(CSRC), "-c", str(CSRC / src), "-o",
               str(obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"--- {src} ---\n{out}")
        elif verbose and out.strip():
            print(out, file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib.with_suffix(".so.tmp")
    cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
