"""The N > 1 host path of bench.py on CPU: two gloo ranks (replicas, weak
scaling) agree on the slowest rank's time, count every rank's units, and draw
disjoint parameter sets.  No GPU, no collective on the data path."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        ms_local = 10.0 + 5.0 * rank                 # rank 1 is the slowest
        ms = bench.max_over_ranks(ms_local, dist)
        value = bench.job_throughput(1000, world, ms)
        first = bench.make_params(rank)[0]            # the rank's first parameter vector
        out[rank] = (ms, value, float(first[0]), float(first[1]))
        bench.barrier(dist)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                      # max over ranks
    assert res[0][1] == res[1][1] == pytest.approx(2000 / 0.015)  # units of both ranks
    assert (res[0][2], res[0][3]) != (res[1][2], res[1][3])    # disjoint seeds


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_throughput(10, 1, 1000.0) == pytest.approx(10.0)
    assert bench.seeds_for(0, 1) != bench.seeds_for(1, 1)
