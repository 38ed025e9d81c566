"""The multi-process side of bench.py on CPU: two gloo ranks, each timing its
share of one record-sharded build; every rank must see the slowest rank's
time, and the rate counts the units of the one build over that time (strong
scaling).  The rank environment is read the way torchrun sets it."""
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
        my_ms = 2.0 + 3.0 * r  # rank 1 is the slow share
        ms = bench.max_over_ranks(my_ms, dist, "cpu")
        rate = bench.strong_rate(1.0e8, ms * 1e-3)
        q.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_share():
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
        assert rate == pytest.approx(1.0e8 / 5.0e-3)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.strong_rate(2.0e8, 0.5) == pytest.approx(4.0e8)


def test_method_flops_follow_the_per_unit_rule():
    """The roofline's algorithmic work: sum over classes of records x half-sphere
    points x (4L + 14), times the densities, independent of the form."""
    import bench

    info = {"ng_half": 10, "pairs_by_class": [3, 2, 1, 0, 1], "n1_table": 13}
    assert bench.walk_flops(info, 2) == 2 * 10 * (3 * 14 + 2 * 18 + 1 * 22 + 1 * 30)
    assert bench.walk_emulation_ops(info, 1) == 10 * (3 * 72 + 2 * 110 + 1 * 148 + 1 * 224)
