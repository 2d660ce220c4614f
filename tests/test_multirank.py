"""The N-rank bench path on CPU ranks (gloo, world size 2): independent
replicas, a barrier, the slowest rank's time and the sum of all ranks'
tuples (no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    dist.barrier()
    ms, tuples = bench.combine_ranks(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist, torch.device("cpu"))
    q.put((rank, ms, tuples))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_max_time_sum_tuples():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=100) for _ in ps)
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, ms, tuples in out:
        assert ms == 150.0 and tuples == 3000.0
