"""Allocation-free residual entry point (nsk_rhs_static_scratch).

Some callers cannot allocate device memory: a plugin inside a host application
that owns all device memory through its own pool, or a loop that must not
trigger the device-wide synchronisation that cudaMalloc / cudaFree imply. For
them the library offers a residual whose scratch lives in a fixed file-scope
device array. These checks call it through the C ABI on caller-owned device
tensors and compare it with the context-based nsk_rhs, on two calls in a row
with different states (the shared scratch keeps the previous call's contents,
so the second call shows that nothing stale leaks into its result), and check
that sizes beyond the array, and aliased input and output arrays, are rejected.
Both paths run the same stage kernels with the same parameters, so their
residuals must agree bit for bit (any difference would be a stale scratch value
or a parameter set differently); the oracle's residual tolerance is checked as
well. This file is collected last.
"""
import numpy as np
import pytest

from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu

CASE = dict(dim=3, nelem=(6, 5, 4), N=3, node_type=nsk.NSK_NODES_GAUSS, lo=(0.0, 0.0, 0.0), hi=(1.0, 0.8, 1.2))
PRM = dict(T=0.85, kappa=1e-3, alpha=1e3, beta=1e-3, mu=2e-2)


def _context_rhs(U):
    s = nsk.Solver(CASE["dim"], CASE["nelem"], CASE["N"], list(CASE["lo"]), list(CASE["hi"]), CASE["node_type"])
    s.set_params(**PRM)
    s.set_state(U)
    R = s.rhs()
    s.close()
    return R


def test_static_scratch_matches_context_rhs(gpu):
    import torch

    import oracle as O
    from tolerances import rhs_tolerance  # the residual parity tolerance of the other GPU tests

    o = O.Oracle(CASE["dim"], CASE["nelem"], CASE["lo"], CASE["hi"], CASE["N"], CASE["node_type"], **PRM)
    stream = torch.cuda.current_stream()
    for seed in (31, 32):  # two calls in a row, different states
        U = inputs.random_state(o.shape, seed=seed)
        Ud = torch.from_numpy(U).to(gpu)
        Rd = torch.full_like(Ud, float("nan"))
        code = nsk.nsk_rhs_static_scratch(CASE["dim"], CASE["nelem"], CASE["lo"], CASE["hi"], CASE["N"],
                                          CASE["node_type"], PRM["T"], PRM["kappa"], PRM["alpha"], PRM["beta"],
                                          PRM["mu"], Ud, Rd, stream.cuda_stream)
        assert code == nsk.NSK_OK, nsk.error_string(code)
        torch.cuda.synchronize()
        R_static = Rd.cpu().numpy()
        R_ctx = _context_rhs(U)
        assert np.array_equal(R_static, R_ctx), (seed, float(np.abs(R_static - R_ctx).max()))
        Ro = o.rhs(U)
        tol = rhs_tolerance(o, U, Ro)
        for v in range(o.nvar):
            err = float(np.abs(R_static[v] - Ro[v]).max())
            assert err <= tol[v], (seed, v, err, tol[v])


def test_static_scratch_rejects_oversized_meshes_and_aliasing(gpu):
    import torch

    cap = nsk.load_library().nsk_static_scratch_bytes()
    assert cap == 64 << 20
    # 3D, N = 3 needs 16512 bytes per element: 20^3 elements do not fit in 64 MiB. The arrays are
    # allocated at the full size the mesh needs, so even a regressed size check could not make the
    # kernels reach past them.
    n = 5 * 20**3 * 64
    U = torch.full((n,), 1.2, dtype=torch.float64, device=gpu)
    R = torch.zeros(n, dtype=torch.float64, device=gpu)
    code = nsk.nsk_rhs_static_scratch(3, (20, 20, 20), (0, 0, 0), (1, 1, 1), 3, 0, 0.85, 1e-4, 1e3, 1e-3, 1e-3,
                                      U, R)
    assert code == nsk.NSK_ERR_ARG
    # a mesh that fits, with the output aliasing the input: rejected before any launch
    m = 5 * 4**3 * 64
    code = nsk.nsk_rhs_static_scratch(3, (4, 4, 4), (0, 0, 0), (1, 1, 1), 3, 0, 0.85, 1e-4, 1e3, 1e-3, 1e-3,
                                      U[:m], U[:m])
    assert code == nsk.NSK_ERR_ARG
