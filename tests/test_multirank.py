"""Host logic of the N-GPU bench path on CPU: world_size-2 gloo ranks run the replica
aggregation bench.py uses (max of the ranks' times, sum of their work)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    t, u = bench.aggregate_replicas(1.5 + rank, 1000 * (rank + 1), dist, "cpu")
    q.put((r, ws, local, t, u))
    dist.destroy_process_group()


def test_replica_aggregation_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, ws, local, t, u) in enumerate(res):
        assert rank == r and ws == 2 and local == r
        assert t == 2.5 and u == 3000.0            # slowest rank, total work
