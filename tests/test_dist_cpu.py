"""The multi-process path of bench.py (replicas, one per GPU) on CPU ranks.

Each rank runs an independent replica; the only cross-rank steps are the
barrier around the timed region and the max over ranks of the elapsed time.
Two gloo ranks check both.
"""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch

    import bench

    r, w, local = bench.dist_init()
    assert (r, w, local) == (rank, world, rank)
    bench.dist_barrier(w)
    t = bench.dist_max(1.5 + rank, w, torch.device("cpu"))
    results[rank] = t
    bench.dist_barrier(w)
    bench._PG.destroy_process_group()


def test_replica_barrier_and_max_over_ranks():
    import torch
    import torch.multiprocessing as mp

    if torch.cuda.is_available():
        pytest.skip("CPU-only test (bench uses NCCL when a GPU is present)")
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(results) == {0: 2.5, 1: 2.5}
