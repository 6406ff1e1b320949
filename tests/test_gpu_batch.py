"""Stage schedules, autotuner and batched persistent execution.

Every schedule (block size 128/256, face flux separate or fused into the volume
kernel) evaluates the same per-node arithmetic, so results must agree bit for
bit. A batch of uneven 3D instances (different meshes, N = 3 and 4) advanced by
the persistent cooperative kernel must reproduce, bit for bit, each instance
stepped alone; the bounded grid-barrier wait must end with NSK_ERR_TIMEOUT
(not a hang) when the barrier is made unreachable, leaving the batch usable.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs, nsk

pytestmark = pytest.mark.gpu

PRM = dict(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3)


def _state(s, seed):
    """In-range random state (these coarse test meshes cannot resolve a 0.02-wide interface)."""
    return inputs.random_state(s.shape, seed=seed)


@pytest.mark.parametrize("precision", [nsk.NSK_FP64, nsk.NSK_FP32_MIXED])
@pytest.mark.parametrize("dim,ne,N", [(3, (5, 4, 3), 2), (3, (5, 4, 3), 3), (3, (5, 4, 3), 4), (3, (3, 2, 3), 5),
                                      (2, (7, 5), 3), (2, (6, 3), 5), (1, (9,), 3), (1, (5,), 1)])
def test_schedules_are_bit_identical(gpu, precision, dim, ne, N):
    """Separate face pass, face fluxes in the volume kernel, the lean two-launch stage (the
    lifting recomputed on chip), the single-block schedule (where the mesh fits one block; the
    separate face pass elsewhere) and the line-per-thread kernels (FP32 3D N = 3; the separate face
    pass elsewhere), at both block sizes: the same bits."""
    s = nsk.Solver(dim, ne, N, [0] * dim, [1] * dim, 0, precision)
    s.set_params(**PRM)
    U = _state(s, 1)
    results = []
    for tpb in (128, 256):
        for fused in (0, 1, 2, 3, 4):
            s.set_schedule(tpb, fused)
            s.set_state(U)
            R = s.rhs()
            s.step(1e-6, 2)
            results.append((R, s.get_state()))
    for R, Us in results[1:]:
        assert np.array_equal(R, results[0][0])
        assert np.array_equal(Us, results[0][1])
    s.close()


@pytest.mark.parametrize("precision", [nsk.NSK_FP64, nsk.NSK_FP32_MIXED])
@pytest.mark.parametrize("fused", [0, 1, 2, 4])
def test_volume_kernel_traces_equal_a_prolongation_pass(gpu, precision, fused):
    """Inside one nsk_step call every stage after the first takes the face traces that the
    previous stage's volume kernel wrote; a call starts with a prolongation pass. Four steps
    in one call must therefore equal four calls of one step, bit for bit."""
    s = nsk.Solver(3, (5, 4, 3), 3, [0, 0, 0], [1, 1, 1], 0, precision)
    s.set_params(**PRM)
    s.set_schedule(256, fused)
    U = _state(s, 5)
    s.set_state(U)
    s.step(1e-6, 4)
    one_call = s.get_state()
    s.set_state(U)
    for _ in range(4):
        s.step(1e-6, 1)
    assert np.array_equal(s.get_state(), one_call)
    s.set_state(U)
    s.step(-0.5, 3)  # adaptive dt between steps, traces carried across them
    a = s.get_state()
    s.set_state(U)
    for _ in range(3):
        s.step(-0.5, 1)
    assert np.array_equal(s.get_state(), a)
    s.close()


def test_autotune_keeps_state(gpu):
    s = nsk.Solver(3, (8, 8, 8), 3, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP32_MIXED)
    s.set_params(**PRM)
    U = _state(s, 2)
    s.set_state(U)
    before = s.get_state()
    tpb, fused, ms = s.autotune()
    assert tpb in (128, 256) and ms > 0
    assert s.get_schedule() == (tpb, fused)
    assert np.array_equal(s.get_state(), before)
    s.close()


def _instances(precision):
    specs = [((6, 5, 4), 3, 10), ((4, 4, 4), 4, 11), ((7, 3, 5), 3, 12), ((3, 5, 4), 4, 13)]
    out = []
    for ne, N, seed in specs:
        s = nsk.Solver(3, ne, N, [0, 0, 0], [1, 1, 1], 0, precision)
        s.set_params(**PRM)
        out.append((s, _state(s, seed)))
    return out


@pytest.mark.parametrize("precision", [nsk.NSK_FP32_MIXED, nsk.NSK_FP64])
@pytest.mark.parametrize("adaptive", [False, True])
def test_batch_equals_solo_runs(gpu, precision, adaptive):
    solo = _instances(precision)
    expect = []
    for s, U in solo:
        s.set_state(U)
        if adaptive:
            s.step(-0.5, 3)
        else:
            dt = s.compute_dt(0.5)
            s.step(dt, 3)
        expect.append(s.get_state())
        s.close()
    inst = _instances(precision)
    for s, U in inst:
        s.set_state(U)
        s.compute_dt(0.5)
    # the instances' own schedules, used by the batch schedule fused_face = 5
    for (s, _), sched in zip(inst, ((128, 4), (256, 1), (256, 0), (128, 1))):
        s.set_schedule(*sched)
    b = nsk.Batch([s for s, _ in inst])
    for tpb, fused, persistent in ((256, True, 1), (128, False, 1), (256, False, 0), (128, True, 0), (256, False, 2),
                                   (128, True, 2), (256, 2, 2), (128, 2, 2), (256, 4, 2), (128, 4, 2), (256, 5, 2)):
        for s, U in inst:
            s.set_state(U)
            s.compute_dt(0.5)
        b.set_schedule(tpb, fused, persistent)
        ms = b.step(3, cfl=0.5 if adaptive else 0.0, timings=True)
        assert len(ms) == 3 and all(m > 0 for m in ms)
        for (s, _), want in zip(inst, expect):
            assert np.array_equal(s.get_state(), want)
    b.close()
    for s, _ in inst:
        s.close()



@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_batch_per_instance_latency(gpu, persistent):
    """Per-instance step latencies (nsk_batch_step's per_instance_latency_ms): one value per step
    and instance, positive and within the step's wall time; the instance schedule finishes the
    instances of each of its four streams one after another (instance i on stream i mod 4:
    non-decreasing along each stream), a single launch finishes all
    of them together. The stamps do not change the results: the states equal those of a run
    without them, bit for bit."""
    inst = _instances(nsk.NSK_FP32_MIXED)
    for s, U in inst:
        s.set_state(U)
        s.compute_dt(0.5)
    b = nsk.Batch([s for s, _ in inst])
    b.set_schedule(256, False, persistent)
    b.step(2)
    plain = [s.get_state() for s, _ in inst]
    for s, U in inst:
        s.set_state(U)
        s.compute_dt(0.5)
    ms, lat = b.step(2, timings=True, latencies=True)
    assert lat.shape == (2, len(inst))
    for (s, _), want in zip(inst, plain):
        assert np.array_equal(s.get_state(), want)
    for k in range(2):
        assert (lat[k] > 0).all() and (lat[k] <= ms[k] * 1.001 + 1e-3).all(), (lat[k], ms[k])
        if persistent == 2:
            for j in range(4):
                assert (np.diff(lat[k][j::4]) >= 0).all(), lat[k]
        else:
            assert lat[k].max() - lat[k].min() <= 0.05 * lat[k].max() + 5e-3, lat[k]
    b.close()
    for s, _ in inst:
        s.close()

def test_batch_autotune_graph_and_launch_count(gpu):
    inst = _instances(nsk.NSK_FP32_MIXED)
    for s, U in inst:
        s.set_state(U)
        s.compute_dt(0.5)
    b = nsk.Batch([s for s, _ in inst])
    tpb, fused, persistent, ms = b.autotune()
    assert tpb in (128, 256) and persistent in (0, 1, 2) and ms > 0 and b.get_schedule() == (tpb, fused, persistent)
    assert fused in (0, 1) or (fused in (2, 4, 5) and persistent == 2)
    # separate face schedule: one prolongation launch per call, then per stage the persistent
    # kernel, or lifting, face and volume launches (the volume phase writes the next traces)
    for persistent, per_stage in ((1, 1), (0, 3), (2, 3 * len(inst))):
        b.set_schedule(256, False, persistent)
        n0 = b.launch_count
        b.step(2)
        assert b.uses_graph
        assert b.launch_count - n0 == 1 + 2 * 5 * per_stage
    b.set_schedule(256, True, False)  # fused face flux: prolongation, lifting, volume per stage
    n0 = b.launch_count
    b.step(2)
    assert b.launch_count - n0 == 2 * 5 * 3
    # the lean stage per instance: one prolongation per step, then lifting and volume per stage
    b.set_schedule(256, 2, 2)
    n0 = b.launch_count
    b.step(2)
    assert b.launch_count - n0 == 2 * len(inst) * (1 + 5 * 2)
    # the line kernels (N = 3 instances; the others the separate face pass): as the separate pass
    b.set_schedule(128, 4, 2)
    n0 = b.launch_count
    b.step(2)
    assert b.launch_count - n0 == 1 + 2 * 5 * 3 * len(inst)
    with pytest.raises(nsk.NskError):
        b.set_schedule(256, 2, 1)  # the lean stage runs under the instance schedule only
    with pytest.raises(nsk.NskError):
        b.set_schedule(256, 4, 0)  # so do the line kernels
    with pytest.raises(nsk.NskError):
        b.set_schedule(256, 5, 1)  # and the instances' own schedules
    b.close()
    for s, _ in inst:
        s.close()


def test_batch_barrier_wait_is_bounded(gpu):
    """A barrier that can never complete ends every block's wait after the bound and
    reports NSK_ERR_TIMEOUT; the batch then steps normally again."""
    import time

    inst = _instances(nsk.NSK_FP32_MIXED)[:2]
    for s, U in inst:
        s.set_state(U)
        s.compute_dt(0.5)
    b = nsk.Batch([s for s, _ in inst])
    b.set_schedule(256, False, True)
    b.set_timeout(0.05)
    b._test_hook_block_barrier()
    t0 = time.perf_counter()
    with pytest.raises(nsk.NskError) as ei:
        b.step(1)
    assert ei.value.code == nsk.NSK_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    for s, U in inst:
        s.set_state(U)
        s.compute_dt(0.5)
    b.set_timeout(1.0)
    b.step(1)
    b.close()
    for s, _ in inst:
        s.close()


@pytest.mark.parametrize("tpb", [128, 256])
def test_line_schedule_on_a_droplet_collision(gpu, tpb):
    """The line-per-thread FP32 kernels on a 16^3 head-on droplet collision (256 or 512 blocks,
    the interfaces crossing element lines in every direction): the residual, the state after 20
    steps and the diagnostics equal the separate face pass bit for bit."""
    rv, rl, _ = O.maxwell(0.85)
    runs = []
    for fused in (0, 4):
        s = nsk.Solver(3, (16, 16, 16), 3, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP32_MIXED)
        s.set_params(**PRM)
        s.set_schedule(tpb, fused)
        v = inputs.collision_velocity(40.0, 0.2, 1e-4, rv, rl)
        s.set_state(inputs.head_on_collision(s.node_coords(), v, 0.2, rho_vap=rv, rho_liq=rl, kappa=1e-4))
        R = s.rhs()
        s.step(-0.5, 20)
        runs.append((R, s.get_state(), s.diagnostics()))
        s.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
