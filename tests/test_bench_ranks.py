"""The benchmark's multi-rank host logic on CPU with the gloo backend
(world size 2): the step time is the maximum over ranks, the reported value
counts every rank's units, and only rank 0 runs the reference arm."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_max = bench.max_over_ranks(times[rank], world, device="cpu")
    dist.barrier()
    rate = bench.whole_job_rate(world, 1000, 10, t_max)
    # the reference arm returns without work on ranks other than 0
    skipped = None
    if rank != 0:
        class A:  # only the fields the arm reads before returning
            workload, steps, warmup, gpus = "pile_small", 1, 0, world
        skipped = bench.reference_arm(A(), rank, world) is None
    out.put((rank, t_max, rate, skipped))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.25, 2.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, rate, skipped in res:
        assert t_max == 2.5                      # the slowest rank sets the time
        assert rate == 2 * 1000 * 10 / 2.5       # units of both ranks
    assert res[1][3] is True                     # rank 1 runs no reference work
