"""bench.py's multi-rank arithmetic on CPU (gloo, world size 2): every rank solves its own
copies (replicas only), the job time is the slowest rank's time and the job's units are the
sum over ranks."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = bench.dist_env()
    t, u = bench.aggregate(elapsed_s=1.0 + rank, units=3.0 + rank, ws=ws)
    out.put((r, ws, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ws, t, u in got:
        assert ws == 2
        assert t == pytest.approx(2.0)  # slowest rank
        assert u == pytest.approx(7.0)  # 3 + 4 units
