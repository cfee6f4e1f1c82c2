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
