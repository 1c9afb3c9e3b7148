"""Shared helpers for the GPU tests: move seeded inputs to the device, run the
library through its C ABI, bring pairs back as numpy arrays."""
import numpy as np

import paper_1309_3458_gb300 as ddm


def to_dev(arrays):
    import torch
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays)


def gpu_match(ctx, arrays, flags=0, dev=None):
    """Full match through ddm_count + ddm_match; returns (K, upd, sub)."""
    import torch
    U = dev if dev is not None else to_dev(arrays)
    K = ddm.ddm_count(ctx, *U, flags=flags)
    pairs = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
    K2 = ddm.ddm_match(ctx, *U, pairs, flags=flags)
    assert K2 == K
    p = pairs[:K].cpu().numpy().view(np.uint32)
    return K, p[:, 0].copy(), p[:, 1].copy()


def keys(pu, ps):
    return (pu.astype(np.uint64) << np.uint64(32)) | ps.astype(np.uint64)


def digests_from_pairs(offsets, ps):
    """Per-update order-independent digest (SplitMix64 output summed mod
    2**64) of the matched subscription ids, from a grouped pair list."""
    z = ps.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    cs = np.concatenate([[np.uint64(0)], np.cumsum(z, dtype=np.uint64)])
    return cs[offsets[1:].astype(np.int64)] - cs[offsets[:-1].astype(np.int64)]
