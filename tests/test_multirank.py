"""bench.py's multi-rank bookkeeping on two CPU ranks (gloo): every rank reaches the
barrier and the reported time is the maximum over ranks.  The path itself runs
independent replicas per GPU, with no data exchange."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench

    class Args:
        impl = "reference"  # gloo backend, no GPU

    world, r, _ = bench.dist_init(Args())
    bench.barrier(world)
    v = bench.barrier_max(world, 10.0 * (r + 1))
    q.put((r, world, v))
    dist.destroy_process_group()


def test_two_ranks_report_the_max_over_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert got == [(0, 2, 20.0), (1, 2, 20.0)]
    assert all(p.exitcode == 0 for p in procs)
