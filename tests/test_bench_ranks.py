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


def test_rank_windows_are_disjoint_and_flop_model():
    import bench

    ranks = [bench.windows_for_rank(1.0, 0.05, 8, r) for r in range(4)]
    starts = sorted(x for r in ranks for x in r)
    assert len(starts) == 32 and all(b - a == pytest.approx(0.05) for a, b in zip(starts, starts[1:]))
    assert ranks[1][0] == pytest.approx(1.0 + 8 * 0.05)
    # the amplitude contraction 2 (ov)^2 Q per half-vector dominates the per-vector work
    o, v, Q = 128, 512, 1536
    per_vec = bench.sigma_flops_per_vector(o, v, Q)
    ladder = 2 * 2.0 * (o * v) ** 2 * Q
    assert ladder < per_vec < 1.05 * ladder
    assert bench.tgen_flops(o, v, Q) == 2.0 * Q * (o * v) ** 2
    assert bench.step_flops(o, v, Q, 10, 2) == 10 * per_vec + 2 * bench.tgen_flops(o, v, Q)


def test_window_batches_in_turn_and_together():
    import bench

    big = bench.WORKLOADS["dot-256x1024x3072"]
    assert bench.window_batches(big) == [[0], [1], [2], [3]]
    batched = bench.WORKLOADS["batched-128x512x1536"]
    assert bench.window_batches(batched) == [list(range(8))]
    # windows taken in turn, wrapping round; one batch restarts itself
    seq, b = [], 0
    for _ in range(6):
        seq.append(b)
        b = bench.next_batch(b, 4)
    assert seq == [0, 1, 2, 3, 0, 1]
    assert bench.next_batch(0, 1) == 0
    assert bench.DEFAULT_WORKLOAD == "dot-256x1024x3072" and not big["full_solve"]


def test_reference_arm_line_shape():
    """The reference arm (the oracle on the host cores) prints the contract's line: same metric,
    unit and config as the GPU arm, impl reference, its own cpu_baseline and an e2e with no
    copies; ranks other than 0 do no work."""
    import argparse
    import json

    import bench

    args = argparse.Namespace(workload=bench.DEFAULT_WORKLOAD, steps=1, warmup=0)
    assert bench.run_reference(args, 2, 1) is None
    line = bench.run_reference(args, 1, 0)
    json.dumps(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "TFLOP/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["value"] > 0
    assert line["config"]["workload"] == bench.DEFAULT_WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == dict(value=line["value"], unit="TFLOP/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
