"""Replica aggregation over 2 ranks with gloo on CPU (the N > 1 bench path)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2009_01287_gb300 import replicas
    secs, dofit = replicas.aggregate([1.0 + rank, 5.0 - rank], 100.0 * (rank + 1))
    out[rank] = (secs, dofit)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_gloo():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        secs, dofit = out[r]
        assert secs == [2.0, 5.0]          # max over ranks, entry by entry
        assert dofit == 300.0              # sum over ranks


def test_single_process_identity():
    from paper_2009_01287_gb300 import replicas
    assert replicas.aggregate([3.0], 7.0) == ([3.0], 7.0)
