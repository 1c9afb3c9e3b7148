"""Sharded matching across ranks: the host logic on CPU (gloo, world size 2).

One problem's update set is split into contiguous id ranges, the
subscriptions are broadcast from rank 0, every rank matches its range, the
pair counts are all-gathered into global offsets and the shards gathered on
rank 0.  No GPU is used: each rank's local matcher here is the CPU oracle's
interval tree matching (Algs. 4-5) with the shard's first id added, which is
what the library's update-id base does on the GPU.  The gathered pairs must
equal, element by element, the oracle's pairs for the whole problem.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1309_3458_gb300 import sharded as S
from paper_1309_3458_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("m,world", [(0, 1), (5, 1), (10, 3), (7, 8), (1000, 7), (2, 2)])
def test_shard_bounds_cover_the_update_ids(m, world):
    b = S.shard_bounds(m, world)
    assert len(b) == world
    assert b[0][0] == 0 and b[-1][1] == m
    for (b0, e0), (b1, e1) in zip(b, b[1:]):
        assert e0 == b1
    sizes = [e - s for s, e in b]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    assert sum(sizes) == m


def test_exclusive_prefix():
    assert S.exclusive_prefix([]) == [0]
    assert S.exclusive_prefix([3, 0, 5]) == [0, 3, 3, 8]


def _rank(rank, world, port, name, out):
    import torch
    import torch.distributed as tdist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ulo, uhi, slo, shi = W.make(name, 0.004 if name.startswith("clustered") else 1.0)
    # the subscriptions live on rank 0 only; the broadcast replicates them
    sl = torch.from_numpy(slo.copy()) if rank == 0 else torch.zeros(slo.shape, dtype=torch.float32)
    sh = torch.from_numpy(shi.copy()) if rank == 0 else torch.zeros(shi.shape, dtype=torch.float32)
    S.broadcast_set(sl, sh, src=0)
    assert np.array_equal(sl.numpy(), slo) and np.array_equal(sh.numpy(), shi)
    m = ulo.shape[1]
    b, e = S.shard_bounds(m, world)[rank]
    k, pu, ps = oracle.itm_pairs(np.ascontiguousarray(ulo[:, b:e]), np.ascontiguousarray(uhi[:, b:e]),
                                 sl.numpy(), sh.numpy())
    local = torch.from_numpy(np.stack([pu.astype(np.int64) + b, ps.astype(np.int64)], axis=1)
                             .astype(np.int32))
    counts = S.exchange_counts(k)
    pre = S.exclusive_prefix(counts)
    got = S.gather_shards(local, counts, dst=0)
    if rank == 0:
        out["got"] = got.numpy().copy()
        out["counts"] = counts
        out["pre"] = pre
    tdist.barrier()
    tdist.destroy_process_group()


@pytest.mark.parametrize("name", ["uniform_d1_N1e4_a1", "clustered_d3_N1e7_a100"])
def test_two_ranks_gather_the_single_rank_pairs(name):
    import oracle
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), name, out), nprocs=world, join=True)
    ulo, uhi, slo, shi = W.make(name, 0.004 if name.startswith("clustered") else 1.0)
    K, pu, ps = oracle.itm_pairs(ulo, uhi, slo, shi)
    got = out["got"]
    assert sum(out["counts"]) == K and out["pre"][-1] == K and K > 0
    assert got.shape == (K, 2)
    assert np.array_equal(got[:, 0].astype(np.uint32), pu)
    assert np.array_equal(got[:, 1].astype(np.uint32), ps)
    # rank 1's shard starts where rank 0's pairs end
    m = ulo.shape[1]
    b1 = S.shard_bounds(m, world)[1][0]
    assert out["pre"][1] == int(np.searchsorted(pu, b1))
