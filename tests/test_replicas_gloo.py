"""The multi-process path of bench.py on CPU: two gloo ranks (no GPU).

On several GPUs the benchmark runs independent replicas, one problem per
rank with its own seeds, and reports the slowest rank's time per step; the
only collective is one all-reduce on the timing.
"""
import os
import socket

import pytest

import bench
import synthetic as sy


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.5, 2.5][rank]
        out[rank] = bench.max_over_ranks(local, world, torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    out = mp.Manager().dict()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == 2.5 and out[1] == 2.5


def test_single_rank_needs_no_process_group():
    torch = pytest.importorskip("torch")
    assert bench.max_over_ranks(3.25, 1, torch.device("cpu")) == 3.25


def test_replica_seeds_are_independent_per_rank():
    w = sy.WORKLOADS[bench.DEFAULT_WORKLOAD]
    s0, s1 = bench.replica_seeds(w, 0), bench.replica_seeds(w, 1)
    assert s0["gauge"] == w.gauge_seed and s0["source"] == w.source_seed and s0["subspace"] == w.subspace_seed
    for k in s0:
        assert s0[k] != s1[k]
    # distinct streams across ranks and roles
    assert len({v for r in range(4) for v in bench.replica_seeds(w, r).values()}) == 16
