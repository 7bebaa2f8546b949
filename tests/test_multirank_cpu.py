"""The multi-rank path of bench.py on CPU: two gloo ranks (the benchmark runs one
independent replica per GPU, with no collective on the data path; only the timing is
reduced across ranks)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import json
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 100 (r + 1) units in 1 + r seconds
        value, slowest = bench.aggregate_over_ranks(100.0 * (rank + 1), 1.0 + rank, world)
        pts = bench.rank_points(rank, 16)
        gathered = [None] * world
        dist.all_gather_object(gathered, pts)

        class A:
            workload = "single_large"
            steps, warmup, gpus = 1, 0, world
        ref = bench.run_reference(A, rank) if rank != 0 else "rank 0 runs it"
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(dict(value=value, slowest=slowest, points=gathered, ref=ref), f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard(tmp_path):
    torch = pytest.importorskip("torch")
    import json

    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        # all units over the slowest rank's time, on every rank
        assert r["value"] == pytest.approx((100 + 200) / 2.0)
        assert r["slowest"] == 2.0
        # the batched workload's points are disjoint across ranks
        a, b = r["points"]
        assert not set(a) & set(b) and len(a) == len(b) == 16
    # the reference arm runs on rank 0 only: the other ranks return at once
    assert res[1]["ref"] is None


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_over_ranks(50.0, 2.0, 1) == (25.0, 2.0)
