"""The bench's multi-rank host logic with two gloo ranks on the CPU: max-over-ranks timing, whole-job rates, and
the balanced instance split of the batching form (replicas otherwise: no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    from paper_2409_13036_b300 import meshgen as mg
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "timed" 10 + 5 r ms and 100 + r s: every rank sees the slowest
        ms = bench.reduce_over_ranks([10.0 + 5.0 * rank, 100.0 + rank], "max", dist)
        total = bench.reduce_over_ranks([float(rank + 1)], "sum", dist)[0]
        draws = mg.batch_draws()
        parts = bench.partition_instances([(d[0] + 1) ** 3 for d in draws], world)
        out[rank] = {"ms": ms, "sum": total, "parts": parts,
                     "rate": bench.aggregate_rate(world * 30, ms[0])}
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing_and_partition():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        assert res[r]["ms"] == [15.0, 101.0]
        assert res[r]["sum"] == 3.0
        assert res[r]["rate"] == pytest.approx(2 * 30 / 0.015)
    assert res[0]["parts"] == res[1]["parts"]


def test_partition_covers_every_instance_once_and_balances():
    import bench
    from paper_2409_13036_b300 import meshgen as mg
    costs = [(d[0] + 1) ** 3 for d in mg.batch_draws()]
    for world in (1, 2, 3, 4, 8):
        parts = bench.partition_instances(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # largest-first assignment: no rank exceeds the mean by more than the largest instance
        assert max(loads) - sum(loads) / world <= max(costs)
        if world <= 4:
            assert max(loads) / min(loads) < 1.1
    assert bench.partition_instances([5.0, 3.0, 3.0, 1.0], 2) == [[0, 3], [1, 2]]
