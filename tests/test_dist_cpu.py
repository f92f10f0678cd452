"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2).

Ranks solve independent replicas, so the only exchanges are the barrier around the timed region
and the reductions of the timings (max of the step time, sum of the throughput).  The reference
arm runs on rank 0 alone; other ranks return without work.
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


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init()
    bench.barrier(w)
    res = (w, r, local, bench.allreduce(float(r + 1), w, "max"), bench.allreduce(float(r + 1), w, "sum"),
           bench.run_reference(None, w, r) if r != 0 else None)
    bench.barrier(w)
    dist.destroy_process_group()
    out.put((r, res))


def test_two_gloo_ranks_reduce_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        w, rank, local, mx, sm, ref = results[r]
        assert (w, rank, local) == (2, r, r)
        assert mx == 2.0 and sm == 3.0
        assert ref is None   # rank 1 skips the reference arm; rank 0 did not call it here
