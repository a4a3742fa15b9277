"""The replica path of bench.py on CPU: two gloo ranks.

Under torchrun every rank solves its own copy of the workload (the method has
no exchange step between independent solves). The line rank 0 prints must
count the work of all ranks and divide it by the slowest rank's time.
"""
import multiprocessing as mp
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    import bench

    # rank r: times (1 + r, 10 (r + 1)) and work 100 (r + 1)
    mx, sm = bench.reduce_over_ranks(dist, [1.0 + rank, 10.0 * (rank + 1)], [100.0 * (rank + 1)], device="cpu")
    out.put((rank, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_take_the_slowest_rank_and_all_ranks_work():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(2):
        rank, mx, sm = out.get(timeout=120)
        got[rank] = (mx, sm)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        assert got[rank] == ([2.0, 20.0], [300.0])


def test_single_process_returns_the_local_values():
    import bench

    assert bench.reduce_over_ranks(None, [3.0], [7.0]) == ([3.0], [7.0])
