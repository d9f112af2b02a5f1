"""The distributed form's exchange (Sec. 4.4) on CPU ranks (gloo, world
sizes 2 and 3): each rank holds one contiguous sub-vector, computes its local
top-k (here with the oracle, since no GPU takes part), and
``shard.gather_lists`` all-gathers the lists with their lengths and index
bases. On the gathered layout the final top-k is checked two ways against
the oracle's answer over the whole vector:
  * explicit global indices (part_base[p] + local index) merged by the
    oracle's merge definition;
  * the library's merge rule: the plain top-k over the concatenated lists
    with positions as indices (ties to the smallest position), positions
    then mapped to global indices; this is what drtopk_topk_merge computes
    on the GPU, so the test checks that the gathered layout satisfies its
    requirements (rank order, sorted lists, ties across sub-vector borders).
Sub-vectors shorter than k and ties that straddle rank borders are covered.
"""

import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def whole_vector(kind, n):
    rng = np.random.default_rng(77)
    if kind == "few":
        return rng.integers(0, 5, n).astype(np.uint32)
    return rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)


def _rank_main(rank, world, port, cuts, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2109_08219_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for kind in ("few", "rand"):
            full = whole_vector(kind, cuts[-1])
            mine = full[cuts[rank]:cuts[rank + 1]]
            for smallest in (False, True):
                pick = oracle.bottomk if smallest else oracle.topk
                for k in (1, 7, 300, 900):
                    cnt = min(k, mine.size)
                    lk, li = pick(mine, oracle.U32, cnt)
                    kb = torch.zeros(k, dtype=torch.int32)
                    ib = torch.zeros(k, dtype=torch.int32)
                    kb[:cnt] = torch.from_numpy(lk.view(np.int32))
                    ib[:cnt] = torch.from_numpy(li)
                    kc, ic, off, base = shard.gather_lists(kb, ib, cnt, mine.size, k)
                    kc = kc.numpy().view(np.uint32)
                    ic = ic.numpy().astype(np.int64)
                    part = np.searchsorted(off, np.arange(kc.size), side="right") - 1
                    gidx = base[part] + ic
                    kk = min(k, kc.size)
                    rk, ri = pick(full, oracle.U32, kk)
                    # merge by explicit global indices
                    mk, mg = oracle.topk_merge(kc, gidx, oracle.U32, kk, smallest)
                    ok1 = np.array_equal(mk, rk) and np.array_equal(mg, ri.astype(np.int64))
                    # merge by positions in the gathered layout
                    pk, pi = pick(kc, oracle.U32, kk)
                    ok2 = np.array_equal(pk, rk) and np.array_equal(gidx[pi], ri.astype(np.int64))
                    res.append((kind, smallest, k, bool(ok1), bool(ok2),
                                off.tolist(), base.tolist()))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("cuts", [[0, 1500, 2999], [0, 5, 1200, 2400]])
def test_gathered_lists_merge_to_the_whole_answer(cuts):
    world = len(cuts) - 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, cuts, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank, res in results:
        for kind, smallest, k, ok1, ok2, off, base in res:
            assert ok1 and ok2, (rank, kind, smallest, k)
            assert base == cuts[:-1]
            lens = np.diff(cuts)
            assert off == np.concatenate([[0], np.cumsum(np.minimum(k, lens))]).tolist()
