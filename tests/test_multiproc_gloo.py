"""The bench's multi-rank host logic on CPU: two ranks on the gloo backend.

bench.py runs one independent replica per rank (no data-path collective); the
only cross-rank steps are the barrier before timing and the max over ranks of
the timed duration, from which the whole-job rate follows.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch
    import torch.distributed as dist

    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    dist.barrier()
    # rank r "took" 10 + 5 r ms for 3 steps of 1000 entries
    ms = bench.max_over_ranks(torch, 10.0 + 5.0 * r, w, "cpu")
    rate = bench.job_rate(3 * 1000, w, ms / 1e3)
    dist.destroy_process_group()
    q.put((r, w, local, ms, rate))


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    for _, _, _, ms, rate in out:
        assert ms == pytest.approx(15.0)                       # the slower rank's time on both
        assert rate == pytest.approx(2 * 3000 / 0.015)         # both ranks' units over that time


def test_single_rank_needs_no_process_group():
    import torch

    import bench
    assert bench.max_over_ranks(torch, 7.5, 1, "cpu") == 7.5
    assert bench.job_rate(100, 1, 0.5) == 200.0
