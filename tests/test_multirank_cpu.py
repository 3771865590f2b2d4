"""CPU: the benchmark's multi-rank logic over gloo, world size 2.  Every rank evaluates its own
states (no collective on the data path); the only collective is the max of the elapsed times, and
the whole-job value counts every rank's states over the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [3.0, 5.0][rank]
        mx = bench.max_over_ranks(ms, world, torch.device("cpu"))
        val = bench.job_value(world, 10, 512, mx)
        seeds = [bench.rank_seed(rank, s) for s in range(bench.N_INPUT_SETS)]
        q.put((rank, mx, val, seeds))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_states():
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
    (r0, mx0, v0, s0), (r1, mx1, v1, s1) = res
    assert mx0 == mx1 == 5.0
    assert v0 == v1 == pytest.approx(2 * 10 * 512 / 5e-3)
    assert not set(s0) & set(s1)        # disjoint input sets: weak scaling, nothing shared


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, 1, None) == 4.0
    assert bench.job_value(1, 2000, 512, 1000.0) == pytest.approx(1024000.0)
