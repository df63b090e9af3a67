"""The replica (N > 1) timing path of bench.py on CPU: two gloo ranks, the job
time is the slowest rank's, and the whole-job value counts every rank's events."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    q.put((rank, bench.max_over_ranks(local_ms, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_max_over_ranks_single_process():
    pytest.importorskip("torch")
    import bench

    assert bench.max_over_ranks(3.5) == 3.5


def test_oracle_scaling_table_shape_and_invariant():
    """The thread-scaling table (the paper's Tables 1-8 layout) on a tiny run:
    every thread count gives the identical result (the paper's invariant)."""
    import bench

    t = bench.oracle_scaling(threads=[1, 2], runs=2, warmup=(2, 2000), production=(2, 4000))
    assert [r["threads"] for r in t["rows"]] == [1, 2]
    for r in t["rows"]:
        assert r["identical_to_1_thread"]
        assert r["min_s"] <= r["avg_s"] <= r["max_s"]
        assert r["acceleration"] > 0 and r["efficiency"] > 0
