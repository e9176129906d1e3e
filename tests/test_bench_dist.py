"""The multi-rank host logic of bench.py on CPU: two gloo ranks aggregate
units (sum) and time (max over ranks); the batch workload's instances are
split over the ranks by LPT; a single H-LU is replicated."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        v, t = bench.job_throughput(10.0 * (rank + 1), 1.0 + rank, world)
        dist.barrier()
        out.put((rank, v, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_units_and_take_max_time():
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, t in res:
        assert t == 2.0  # the slowest rank's time
        assert v == pytest.approx(30.0 / 2.0)  # all ranks' units over that time


def test_single_rank_is_plain_ratio():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(12.0, 4.0, 1) == (3.0, 4.0)


def _lpt_worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        mine = bench.rank_problems("diffusion2d_batch64", rank, world)
        # every rank reports its instances; the gather is host-side only
        got = [None] * world
        dist.all_gather_object(got, [p.seed for p in mine])
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_batch_instances_partitioned_by_lpt_over_two_gloo_ranks():
    """Two gloo ranks split the 64 instances: each instance on exactly one
    rank, both ranks agree on the split, and the loads (n log2(n)^2) stay
    within the LPT bound max <= 4/3 max(total / ranks, largest instance)."""
    import torch.multiprocessing as mp
    import socket
    sys.path.insert(0, ROOT)
    import bench
    import hmat_synth as hs
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_lpt_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1]
    parts = res[0][1]
    allp = hs.diffusion2d_batch()
    seeds = sorted(p.seed for p in allp)
    assert sorted(parts[0] + parts[1]) == seeds and not set(parts[0]) & set(parts[1])
    cost = {p.seed: bench.instance_cost(p.n) for p in allp}
    loads = [sum(cost[x] for x in part) for part in parts]
    total = sum(cost.values())
    assert max(loads) <= 4.0 / 3.0 * max(total / 2, max(cost.values()))


def test_lpt_partition_small_cases():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.lpt_partition([5.0, 4.0, 3.0, 3.0, 3.0], 2) == [[0, 3], [1, 2, 4]]
    assert bench.lpt_partition([1.0, 2.0], 3) == [[1], [0], []]
    assert bench.lpt_partition([2.0, 2.0, 2.0, 2.0], 1) == [[0, 1, 2, 3]]


def test_single_instance_is_replicated():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_problems("laplace3d_32", 1, 2)[0].n == bench.rank_problems("laplace3d_32", 0, 2)[0].n
    assert len(bench.rank_problems("diffusion2d_batch64", 0, 1)) == 64


def test_traffic_only_for_the_captured_sources(monkeypatch):
    """roofline.traffic comes from an ncu capture of one source tree: it is
    reported while the kernel sources hash the same, and null otherwise."""
    sys.path.insert(0, ROOT)
    import bench
    h = bench.csrc_hash()
    assert len(h) == 16 and h == bench.csrc_hash()
    monkeypatch.setattr(bench, "TRAFFIC", {"laplace3d_32": {"csrc": h, "bytes": 123}})
    assert bench.traffic_per_launch("laplace3d_32") == 123
    monkeypatch.setattr(bench, "TRAFFIC", {"laplace3d_32": {"csrc": "0" * 16, "bytes": 123}})
    assert bench.traffic_per_launch("laplace3d_32") is None
    assert bench.traffic_per_launch("diffusion2d_batch64") is None


def test_config_names_the_workload_and_its_sizes():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(workload="laplace3d_32", precision="mixed", max_rank=0)
    cfg = bench.workload_config(args, bench.rank_problems("laplace3d_32", 0), 1)
    assert cfg["workload"] == "laplace3d_32" and cfg["n"] == 32 ** 3 and cfg["leaf"] == 64 and cfg["eps"] == 1e-4
    assert "flushed" in cfg["l2"] and cfg["parallelism"] == "replicas1"
    args.workload = "diffusion2d_batch64"
    cfg = bench.workload_config(args, bench.rank_problems("diffusion2d_batch64", 0, 2), 2)
    assert cfg["instances"] < 64 and "LPT" in cfg["parallelism"]
