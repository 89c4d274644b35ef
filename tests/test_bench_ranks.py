"""The multi-rank logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

The GPU runs of this build use one GPU, so the torchrun path (N > 1) is covered here
on its host side: the process group from the environment, the largest time over the
ranks, the barrier, and the per-rank batches of independent problems (weak scaling:
distinct batches, rank 0's the single-GPU one).
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init("gloo")
    assert dist is not None and dist.get_rank() == rank and dist.get_world_size() == world
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, 10.0 * (rank + 1) + 0.25, "cpu")
    out.put((rank, m, bench.batch_seed(rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.25, 20.25]       # both ranks see the largest value
    seeds = [r[2] for r in res]
    assert len(set(seeds)) == 2                         # distinct batches per rank


def test_single_process_needs_no_group(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    sys.path.insert(0, ROOT)
    import bench
    from workloads import batched_problems
    import inspect
    assert bench.dist_init("gloo") is None
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    bench.barrier(None)
    # rank 0's batch is the single-GPU batch
    assert bench.batch_seed(0) == inspect.signature(batched_problems).parameters["seed"].default
