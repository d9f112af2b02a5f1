"""Distributed form of the method (Sec. 4.4, "Distributed Dr. Top-k").

The input vector is split into contiguous sub-vectors, one per rank (one
GPU each). Every rank computes the top-k of its own sub-vector with the
single-query path; the lists are gathered on the primary rank, which
computes the final top-k over them with ``drtopk_topk_merge``. The union of
the per-rank lists holds the answer (an element of the global top-k is in
its own sub-vector's top-k), and because every list is sorted by (key,
index) and the lists are concatenated in rank order, the merge keeps the
smallest-global-index tie rule.

The exchange is one all-gather of fixed-size buffers (k keys and k int32
indices per rank, padded when a sub-vector holds fewer than k keys) plus
one all-gather of (list length, sub-vector length) per rank: the gathered
lists land in each rank's own memory before the merge reads them. The
optional exchange of the ranks' thresholds that the paper tried and
disabled (Sec. 4.4) is not built.

This module is plumbing over ``torch.distributed``; all arithmetic of the
method runs in the CUDA library.
"""

import numpy as np


def gather_lists(keys, idx, count, n_local, k, group=None):
    """All-gathers every rank's local top-k list.

    keys, idx: this rank's list in buffers of k entries (only the first
    ``count`` are valid); n_local: the length of this rank's sub-vector.
    Returns, on every rank, (keys_cat, idx_cat, part_off, part_base): the
    valid parts of all lists concatenated in rank order (tensors on the
    buffers' device), the list boundaries (numpy int64, ranks + 1) and each
    rank's global index base (numpy int64: the sub-vectors are contiguous
    and in rank order, so rank r starts at the sum of the lengths before it).
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if keys.numel() != k or idx.numel() != k:
        raise ValueError("list buffers must hold k entries")
    meta = torch.tensor([int(count), int(n_local)], dtype=torch.int64, device=keys.device)
    metas = torch.empty(world * 2, dtype=torch.int64, device=keys.device)
    dist.all_gather_into_tensor(metas, meta, group=group)
    kk = torch.empty(world * k, dtype=keys.dtype, device=keys.device)
    ii = torch.empty(world * k, dtype=idx.dtype, device=idx.device)
    dist.all_gather_into_tensor(kk, keys.contiguous(), group=group)
    dist.all_gather_into_tensor(ii, idx.contiguous(), group=group)
    m = metas.cpu().numpy().reshape(world, 2)
    counts, lens = m[:, 0], m[:, 1]
    if np.any(counts > k) or np.any(counts < 0):
        raise ValueError("list counts out of range")
    part_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    part_base = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    if np.all(counts == k):
        return kk, ii, part_off, part_base
    keys_cat = torch.cat([kk[r * k:r * k + int(counts[r])] for r in range(world)])
    idx_cat = torch.cat([ii[r * k:r * k + int(counts[r])] for r in range(world)])
    return keys_cat, idx_cat, part_off, part_base


def shard_topk(x_local, k, smallest=False, dtype=None, group=None, root=0, stream=None):
    """Top-k of the vector whose rank-ordered sub-vectors are each rank's
    ``x_local`` (a 1-D CUDA tensor). Returns (keys, int64 global indices) on
    ``root`` and None elsewhere. Collective: every rank of the group calls
    it with the same k."""
    import torch
    import torch.distributed as dist
    from . import drtopk_select, drtopk_topk_merge
    n = x_local.numel()
    cnt = min(k, n)
    ok = torch.zeros(k, dtype=x_local.dtype, device=x_local.device)
    oi = torch.zeros(k, dtype=torch.int32, device=x_local.device)
    if cnt > 0:
        lk, li, _ = drtopk_select(x_local, cnt, smallest=smallest, dtype=dtype, stream=stream)
        ok[:cnt] = lk
        oi[:cnt] = li
    keys_cat, idx_cat, part_off, part_base = gather_lists(ok, oi, cnt, n, k, group=group)
    if dist.get_rank(group) != root:
        return None
    total = int(part_off[-1])
    return drtopk_topk_merge(keys_cat, idx_cat, part_off, part_base, min(k, total),
                             smallest=smallest, dtype=dtype, stream=stream)
