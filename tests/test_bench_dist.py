"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
timing scalars are combined across ranks (max of times, sum of evaluations)
and no data-path collective exists; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist = bench.init_dist(world, "gloo")
    mx = bench.max_over_ranks(dist, 100.0 + rank)          # per-rank elapsed ms
    total = bench.sum_over_ranks(dist, 1e9 * (rank + 1))   # per-rank evaluations
    q.put((rank, mx, total, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, total, env in out:
        assert mx == 101.0            # the slowest rank's time
        assert total == 3e9           # all ranks' evaluations
        assert env == (rank, 2, rank)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--gpus", "2"]) == 0   # exits without work


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 5.0) == 5.0 and bench.sum_over_ranks(None, 7.0) == 7.0
    args = bench.parse_args([])
    assert args.gpus == 1 and args.steps >= 1 and args.warmup >= 3


def test_traffic_record_is_used_only_for_its_kernel_source(monkeypatch):
    """roofline.traffic comes from the committed one-pass ncu record only while
    the sensor kernel's sources hash to the digest stored with the counters:
    its DRAM bytes read and written, scaled by the launch's evaluations; for
    any other source it is None."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "sensor_dram_traffic.json")))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: rec["kernel_digest"])
    per_eval = (rec["dram_bytes_read"] + rec["dram_bytes_write"]) / rec["evals"]
    assert bench.measured_traffic(1000, 2048) == per_eval * 1000 * 2048
    assert abs(bench.measured_traffic(1_000_000, 65536) - (rec["dram_bytes_read"] + rec["dram_bytes_write"])) < 1.0
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "not-" + rec["kernel_digest"])
    assert bench.measured_traffic(1000, 2048) is None
