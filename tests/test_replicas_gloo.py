"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the path has no exchange step, so
ranks run independent replicas; the reported time is the maximum over ranks and the work the sum."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = bench.allreduce_max(1.5 + rank, world)          # per-rank step times 1.5 s and 2.5 s
    w = bench.allreduce_sum(10.0 * (rank + 1), world)   # per-rank voxel-iterations 10 and 20
    dist.destroy_process_group()
    q.put((rank, t, w))


def test_replica_reductions_take_max_time_and_sum_work():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, w in out:
        assert t == 2.5 and w == 30.0
