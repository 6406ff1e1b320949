"""The bounds-checking build (libnsk_check.so, -DNSK_BOUNDS_CHECK): its index checks change no
result (the same bits as the regular library on residuals and steps, model II, every schedule,
1D-3D) and, when a test hook points the neighbour strides outside the mesh (possible in that build
only), they catch every access: the call returns NSK_ERR_BOUNDS instead of faulting. The checked
library runs in a child process (NSK_LIBRARY names it)."""
import os
import subprocess
import sys
import textwrap
from pathlib import Path

import numpy as np
import pytest

from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]
CASES = [(3, (5, 4, 3), 3, 0), (3, (4, 3, 3), 2, 1), (3, (3, 4, 2), 3, 2), (2, (7, 5), 4, 0), (1, (9,), 3, 3)]
PRM = dict(T=0.85, kappa=1e-3, alpha=1e3, beta=1e-3, mu=2e-2)

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, sys.argv[1])
    from paper_1912_12059_gb300 import inputs, nsk
    out = {}
    for i, (dim, ne, N, sched) in enumerate(eval(sys.argv[3])):
        s = nsk.Solver(dim, ne, N, [0] * dim, [1] * dim, 0, nsk.NSK_FP64)
        s.set_params(**eval(sys.argv[4]))
        s.set_schedule(256, sched)
        U = inputs.random_state(s.shape, seed=10 + i)
        s.set_state(U)
        out[f"R{i}"] = s.rhs()
        s.step(1e-6, 2)
        out[f"U{i}"] = s.get_state()
        s.close()
    s = nsk.Solver(3, (5, 4, 3), 3, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP64)
    s.set_params(**eval(sys.argv[4]))
    s.set_state(inputs.random_state(s.shape, seed=99))
    out["hook"] = np.array([nsk.load_library().nsk_test_hook_corrupt_neighbours(s.ctx)])
    try:
        s.rhs()
        out["code"] = np.array([0])
    except nsk.NskError as ex:
        out["code"] = np.array([ex.code])
    np.savez(sys.argv[2], **out)
""")


def test_checked_build_same_bits_and_catches_bad_indices(gpu, tmp_path):
    from paper_1912_12059_gb300.build import build_library

    lib = build_library(bounds_check=True)
    res = tmp_path / "checked.npz"
    env = dict(os.environ, NSK_LIBRARY=str(lib))
    r = subprocess.run([sys.executable, "-c", CHILD, str(ROOT), str(res), repr(CASES), repr(PRM)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(res)
    for i, (dim, ne, N, sched) in enumerate(CASES):
        s = nsk.Solver(dim, ne, N, [0] * dim, [1] * dim, 0, nsk.NSK_FP64)
        s.set_params(**PRM)
        s.set_schedule(256, sched)
        U = inputs.random_state(s.shape, seed=10 + i)
        s.set_state(U)
        assert np.array_equal(s.rhs(), got[f"R{i}"]), i
        s.step(1e-6, 2)
        assert np.array_equal(s.get_state(), got[f"U{i}"]), i
        s.close()
    assert int(got["hook"][0]) == nsk.NSK_OK and int(got["code"][0]) == nsk.NSK_ERR_BOUNDS
    # the regular library has no checks: its hook refuses and changes nothing
    s = nsk.Solver(2, (3, 3), 2)
    assert nsk.load_library().nsk_test_hook_corrupt_neighbours(s.ctx) == nsk.NSK_ERR_STATE
    s.close()
