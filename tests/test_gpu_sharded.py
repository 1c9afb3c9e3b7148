"""Sharded matching on the GPU: shards of one problem's update set, matched
one after another in one process (each with its own context, as separate
ranks would), concatenate to exactly the single-call output.

Queries are independent (Section IV, "Parallelizing ITM"), and with the
update-id base set to its first id a shard writes global update ids; the
tree is built from the same subscriptions by the same deterministic build, so
each shard's pairs are the single call's pairs for its range, in the same
order.  The union is also checked against the oracle's pair set.
"""
import numpy as np
import pytest

import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import sharded as S
from paper_1309_3458_gb300 import workloads as W

from .helpers import keys, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    import __graft_entry__
    __graft_entry__.build()
    hs = [ddm.ddm_create(0) for _ in range(4)]
    yield hs
    for h in hs:
        ddm.ddm_destroy(h)


def single(ctx, U):
    import torch
    K = ddm.ddm_count(ctx, *U)
    pairs = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
    assert ddm.ddm_match(ctx, *U, pairs) == K
    return pairs[:K].cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("name,scale,world", [
    ("uniform_d1_N1e4_a1", 1.0, 2),
    ("uniform_d2_N1e6_a100", 0.05, 3),
    ("clustered_d3_N1e7_a100", 0.01, 4),
])
def test_shards_concatenate_to_the_single_call(ctxs, name, scale, world):
    import torch
    import oracle
    arrays = W.make(name, scale)
    U = to_dev(arrays)
    ddm.ddm_set_update_id_base(ctxs[0], 0)
    whole = single(ctxs[0], U)
    m = arrays[0].shape[1]
    parts, counts = [], []
    for r, (b, e) in enumerate(S.shard_bounds(m, world)):
        c = ctxs[r]
        lo = torch.from_numpy(np.ascontiguousarray(arrays[0][:, b:e])).cuda()
        hi = torch.from_numpy(np.ascontiguousarray(arrays[1][:, b:e])).cuda()
        plan = S.plan_shard(c, lo, hi, b, U[2], U[3], rank=r, world=1)
        assert plan.begin == b and plan.end == e
        # chunked by update id through a buffer far smaller than the shard
        buf = torch.empty((max(plan.k_local // 3, 64), 2), dtype=torch.int32, device="cuda")
        got = []
        assert S.write_shard(c, plan, buf, lambda ch, at: got.append(ch.cpu().numpy().copy())) \
            == plan.k_local
        parts.append(np.concatenate(got).view(np.uint32) if got else np.zeros((0, 2), np.uint32))
        counts.append(plan.k_local)
        ddm.ddm_set_update_id_base(c, 0)
    cat = np.concatenate(parts)
    assert np.array_equal(cat, whole)          # same pairs, same order
    pre = S.exclusive_prefix(counts)
    for r, (b, e) in enumerate(S.shard_bounds(m, world)):
        seg = cat[pre[r]:pre[r + 1], 0]
        assert seg.size == 0 or (seg.min() >= b and seg.max() < e)
    K, pu, ps = oracle.itm_pairs(*arrays)
    assert cat.shape[0] == K
    assert np.array_equal(np.sort(keys(cat[:, 0], cat[:, 1])), np.sort(keys(pu, ps)))


def test_update_id_base_on_ordered_writes_and_limits(ctxs):
    import torch
    arrays = W.make("uniform_d2_N1e6_a1", 0.02)
    U = to_dev(arrays)
    c = ctxs[0]
    ddm.ddm_set_update_id_base(c, 0)
    ddm.ddm_build(c, U[2], U[3])
    K = ddm.ddm_plan(c, U[0], U[1])
    m = arrays[0].shape[1]
    ref = torch.empty((K, 2), dtype=torch.int32, device="cuda")
    assert ddm.ddm_write_ordered(c, 0, m, ref) == K
    base = 1_000_000
    ddm.ddm_set_update_id_base(c, base)
    got = torch.empty((K, 2), dtype=torch.int32, device="cuda")
    assert ddm.ddm_write_ordered(c, 0, m, got) == K
    assert torch.equal(got[:, 1], ref[:, 1])
    assert torch.equal(got[:, 0].long(), ref[:, 0].long() + base)
    # the compressed output is subscription ids only: unchanged by the base
    ids = torch.empty(K, dtype=torch.int32, device="cuda")
    assert ddm.ddm_write_ordered_ids(c, 0, m, ids) == K
    assert torch.equal(ids, ref[:, 1])
    # global ids that would pass 2^32 are refused
    ddm.ddm_set_update_id_base(c, (1 << 32) - 5)
    with pytest.raises(ddm.DDMError) as e:
        ddm.ddm_write_ordered(c, 0, m, got)
    assert e.value.code == ddm.DDM_ERR_ARG
    ddm.ddm_set_update_id_base(c, 0)
