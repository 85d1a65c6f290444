"""Multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): every
rank transfers its own body with no data-path collective; the job's step time is
the slowest rank's and the throughput sums all ranks' pairs."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = [4.0, 5.5][rank]
    pairs = [700000, 716130][rank]
    t, total, value = bench.aggregate(step_ms, pairs, world, device="cpu")
    out[rank] = (t, total, value, bench.workload_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_is_max_time_and_total_pairs():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, total, value, seed = out[r]
        assert t == 5.5
        assert total == 700000 + 716130
        assert abs(value - total / 5.5e-3) < 1e-6 * value
    assert out[0][3] != out[1][3]  # independent bodies per rank


def test_body_sharding_is_balanced_and_complete():
    import bench
    sizes = [1000, 200000, 5000, 64000, 12000, 150000, 3000, 90000]
    parts = bench.shard_bodies(sizes, 2)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert bench.shard_bodies(sizes, 1) == [list(range(len(sizes)))]
