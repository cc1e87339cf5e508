"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2):
every rank draws its own instances (no collective on the data path) and the
job throughput is taken over the slowest rank."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2005_01182_gb300 import workloads as W
    sizes = W.batch_sizes(64, seed=bench.rank_seed(rank))
    first = W.embedding_costs(int(sizes[0]), seed=bench.rank_seed(rank) + 1)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    value, ms = bench.job_throughput(local_ms, 64, 10, world, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (int(first.sum()), sizes.tolist()))
    q.put((rank, value, ms, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, gathered in res:
        assert ms == 200.0                       # max over ranks
        assert value == pytest.approx(2 * 64 * 10 / 0.2)
        (s0, z0), (s1, z1) = gathered
        assert s0 != s1 or z0 != z1              # ranks solve different instances
