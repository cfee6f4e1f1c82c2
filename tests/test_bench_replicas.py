"""The benchmark's multi-rank host logic on CPU: two gloo ranks meet at the barriers, agree on
the slowest rank's time, and report the whole-job throughput; the oracle arm runs on rank 0."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rep = bench.Replicas(dist, "cpu")
        rep.barrier()
        ms = rep.max(100.0 + 10.0 * rank)
        rep.barrier()
        out[rank] = (ms, bench.replica_value(32768, ms, world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 110.0
    assert res[0][1] == pytest.approx(2 * 32768 / 0.110)


def test_single_rank_and_reference_rule():
    rep = bench.Replicas(None)
    rep.barrier()
    assert rep.max(3.5) == 3.5
    assert bench.replica_value(1000, 2.0, 1) == pytest.approx(5e5)
    assert bench.reference_runs_here(0, 1) and bench.reference_runs_here(0, 4)
    assert not bench.reference_runs_here(1, 4)


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the CPU oracle, timed on the host cores) prints one JSON line
    with the keys of the GPU arm's line, the same workload config, and its own CPU-baseline
    record; e2e moves no bytes between host and device."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"] == dict(bench.WORKLOAD, parallelism="single")
    assert d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
