"""Multi-rank timing aggregation of bench.py on CPU (gloo, world size 2).

Each rank matches its own update set; the job's time is the slowest rank's
and its pairs are the sum over ranks.  No GPU is used.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, k = bench.job_totals(1.0 + rank, 100 * (rank + 1), world, device="cpu")
    out[rank] = (t, k)
    tdist.barrier()
    tdist.destroy_process_group()


def test_job_totals_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (2.0, 300.0)


def test_job_totals_single_rank():
    import bench
    assert bench.job_totals(1.5, 42, 1) == (1.5, 42.0)
