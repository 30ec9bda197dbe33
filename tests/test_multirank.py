"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) combine their timed
regions as the bench does -- max over ranks, all ranks' work -- with no
data-path collective (each rank runs an independent replica)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    max_ms, value = bench.combine_ranks(local_ms, 1e12, 5, world, dist, "cpu")
    q.put((rank, max_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, value in out:
        assert max_ms == 200.0
        assert value == pytest.approx(2 * 1e12 * 5 / 0.2 / 1e12)


def test_single_rank_combination():
    import bench
    max_ms, value = bench.combine_ranks(250.0, 2e12, 4, 1, None, "cpu")
    assert max_ms == 250.0 and value == pytest.approx(2e12 * 4 / 0.25 / 1e12)
