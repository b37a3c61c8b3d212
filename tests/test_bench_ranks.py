"""Host logic of the N > 1 bench path on CPU: two gloo ranks, max time and summed roots."""

import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, roots = bench.reduce_over_ranks(dist, 100.0 + 50.0 * rank, 8 - rank, "cpu")
    w = bench.window_for_rank(1.0, 0.1, rank)
    q.put((rank, ms, roots, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, roots, w in out:
        assert ms == 150.0 and roots == 15.0
    assert out[0][3] == pytest.approx(1.0) and out[1][3] == pytest.approx(1.1)
