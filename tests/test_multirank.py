"""The multi-process side of bench.py on CPU: two gloo ranks, each a replica
with its own step time; every rank must see the slowest rank's time, and the
whole-job rate counts the units of all replicas over that time.  The rank
environment is read the way torchrun sets it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        my_ms = 2.0 + 3.0 * r  # rank 1 is the slow replica
        ms = bench.max_over_ranks(my_ms, dist, "cpu")
        rate = bench.whole_job_rate(w, 1.0e8, ms * 1e-3)
        q.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(world))
    for r, (rank, w, local, ms, rate) in enumerate(got):
        assert (rank, w, local) == (r, world, r)
        assert ms == pytest.approx(5.0)
        assert rate == pytest.approx(world * 1.0e8 / 5.0e-3)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 2.0e8, 0.5) == pytest.approx(4.0e8)
