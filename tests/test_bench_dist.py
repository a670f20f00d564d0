"""Host logic of the multi-GPU bench path on CPU: two gloo ranks take the
max-over-ranks time, form the whole-job weak-scaling value, and solve
disjoint sources (independent problems, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = 1.5 + rank                      # rank 1 is the slow one
        tmax = bench.barrier_max(t, world)
        out[rank] = (tmax, bench.weak_value(64, world, tmax), bench.rank_source_ids(4, rank))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_value():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == pytest.approx(64 * 2 / 2.5)
    assert set(res[0][2]).isdisjoint(res[1][2]) and res[0][2] == [0, 1, 2, 3] and res[1][2] == [4, 5, 6, 7]


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.barrier_max(3.25, 1) == 3.25
    assert bench.weak_value(64, 1, 2.0) == 32.0
    assert bench.rank_source_ids(3, 0) == [0, 1, 2]
