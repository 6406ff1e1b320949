"""nsk_step_host (the state from host memory, the steps, the state back to host memory) against
nsk_set_state + nsk_step + nsk_get_state: the same kernels in the same order on the same data, so
the same state bit for bit, whether the copies overlap the first and last stages (FP64, 3D, N = 3,
the separate face pass, a z extent of a multiple of 8 elements) or the three calls are made in
turn (any other mesh or schedule)."""
import numpy as np
import pytest

from paper_1912_12059_gb300 import nsk

pytestmark = pytest.mark.gpu


def _solver(ne, precision=nsk.NSK_FP64, N=3):
    """A smooth periodic state: rho = 1 + 0.05 sin sin sin, m = 0.02 (cos 2 pi z, sin 2 pi x,
    cos 2 pi y) rho, c = rho + 1e-3 sin 2 pi (x + y)."""
    s = nsk.Solver(3, ne, N, [0, 0, 0], [1, 1, 1], 0, precision)
    s.set_params(T=0.85, kappa=2.5e-3, alpha=1e2, beta=1e-2, mu=1e-2)
    x, y, z = s.node_coords()
    tp = 2.0 * np.pi
    rho = 1.0 + 0.05 * np.sin(tp * x) * np.sin(tp * y) * np.sin(tp * z)
    U0 = np.stack([rho, 0.02 * np.cos(tp * z) * rho, 0.02 * np.sin(tp * x) * rho, 0.02 * np.cos(tp * y) * rho,
                   rho + 1e-3 * np.sin(tp * (x + y))])
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    s.set_state(U0)
    return s, U0, s.compute_dt(0.3)


def _three_calls(s, U0, dt, nsteps):
    s.set_state(U0)
    s.step(dt, nsteps)
    return s.get_state()


@pytest.mark.parametrize("ne,tpb,nsteps", [((8, 8, 8), 256, 1), ((8, 8, 8), 128, 3), ((6, 4, 16), 256, 2),
                                           ((16, 16, 16), 256, 1)])
def test_overlapped_host_step_equals_the_three_calls(gpu, ne, tpb, nsteps):
    s, U0, dt = _solver(ne)
    s.set_schedule(tpb, 0)
    want = _three_calls(s, U0, dt, nsteps)
    U = U0.copy()
    s.step_host(U, dt, nsteps)                 # in place: the output aliases the input
    assert np.array_equal(U, want)
    out = np.full_like(U0, np.nan)
    s.step_host(U0.copy(), dt, nsteps, out=out)  # separate output
    assert np.array_equal(out, want)
    # after the call the context holds the final state, as after nsk_step
    assert np.array_equal(s.get_state(), want)
    s.close()


def test_pinned_tensors(gpu):
    import torch

    s, U0, dt = _solver((8, 8, 8))
    s.set_schedule(256, 0)
    want = _three_calls(s, U0, dt, 2)
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    s.step_host(Uh, dt, 2)
    assert np.array_equal(Uh.numpy(), want)
    s.close()


@pytest.mark.parametrize("ne,precision,sched", [((6, 6, 6), nsk.NSK_FP64, (256, 0)),        # z not a multiple of 8
                                                ((8, 8, 8), nsk.NSK_FP64, (256, 1)),        # fused face schedule
                                                ((8, 8, 8), nsk.NSK_FP32_MIXED, (128, 4))])  # FP32 operator
def test_other_meshes_and_schedules_take_the_three_calls(gpu, ne, precision, sched):
    s, U0, dt = _solver(ne, precision)
    s.set_schedule(*sched)
    want = _three_calls(s, U0, dt, 2)
    U = U0.copy()
    s.step_host(U, dt, 2)
    assert np.array_equal(U, want)
    s.close()


def test_rejects_bad_arguments(gpu):
    s, U0, dt = _solver((8, 8, 8))
    with pytest.raises(nsk.NskError):
        s.step_host(U0.copy(), -dt, 1)
    with pytest.raises(nsk.NskError):
        s.step_host(U0.copy(), dt, 0)
    s.close()


def test_full_size_in_the_benchmark_configuration(gpu):
    """The 3D head-on collision at 64^3, N = 3, FP64 with the separate face pass of 256 threads
    (the benchmark's workload and schedule; slabs of 8 z planes): one step through
    nsk_step_host equals the three calls bit for bit."""
    import torch

    import bench

    wl = bench.workload_by_name("collision3d")
    s = nsk.Solver(wl.dim, wl.nelem, wl.N, list(wl.lo[:wl.dim]), list(wl.hi[:wl.dim]), wl.node_type, nsk.NSK_FP64)
    s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    U0 = np.ascontiguousarray(wl.initial_state(s.node_coords()), dtype=np.float64)
    s.set_state(U0)
    s.set_schedule(256, 0)
    dt = s.compute_dt(wl.cfl)
    want = _three_calls(s, U0, dt, 1)
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    s.step_host(Uh, dt, 1)
    assert np.array_equal(Uh.numpy(), want)
    s.close()
