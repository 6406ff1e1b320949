"""The multi-rank path of bench.py on the CPU (two gloo ranks, no GPU): the whole-job
aggregation takes the slowest rank's times and the sum of all ranks' nodes, and the reference
arm prints only on rank 0 (the other ranks exit without work)."""
import io
import os
import sys
from contextlib import redirect_stdout
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, e2e, nodes = bench.aggregate_ranks(10.0 + rank, 0.5 * (world - rank), 1000 * (rank + 1), world, "cpu")
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.run_reference(bench.argparse.Namespace(gpus=world, steps=0, warmup=0), None, rank, world) \
                if rank != 0 else 0
        out.put((rank, ms, e2e, nodes, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, nodes, rc, printed in res:
        assert ms == 11.0 and e2e == 1.0 and nodes == 3000.0
        assert rc == 0
        if rank == 1:
            assert printed == ""  # non-zero ranks of the reference arm print nothing
