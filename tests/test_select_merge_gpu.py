"""drtopk_select (largest and smallest criteria, Sec. 1 / Sec. 2) and
drtopk_topk_merge (the distributed form's final step, Sec. 4.4) against
the CPU oracle, element by element.

Smallest-k runs the same kernels on complemented order-mapped keys, so the
cases span the same paths as the largest criterion: several tiles and a
ragged tail, tie-heavy inputs reaching the tie walk, k above 4096 (radix
sort of the outputs), float specials. The merge splits one array into
shards (views at arbitrary offsets, so unaligned shard starts occur), runs
drtopk_select on each, concatenates the lists in shard order and merges;
the answer must equal the oracle's top-k of the whole array, including
ties that straddle shard borders and shards shorter than k. Global index
bases above 2^31 are checked against the oracle's merge definition.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu

DT = {"u32": oracle.U32, "i32": oracle.I32, "f32": oracle.F32}
TDT = {"u32": torch.int32, "i32": torch.int32, "f32": torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def host_bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def to_dev(bits, dt):
    return torch.from_numpy(bits.view(np.int32).copy()).view(TDT[dt]).cuda()


def gen(kind, n, seed, dt):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        b = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    elif kind == "few":
        b = rng.integers(0, 5, n).astype(np.uint32) * np.uint32(0x01010101)
    elif kind == "equal":
        b = np.full(n, 0x9E3779B9, np.uint32)
    elif kind == "asc":
        b = (np.arange(n, dtype=np.uint64) * 4 + rng.integers(0, 4, n)).astype(np.uint32)
    elif kind == "desc":
        b = ~(np.arange(n, dtype=np.uint64) * 4 + rng.integers(0, 4, n)).astype(np.uint32)
    elif kind == "normal":
        b = rng.standard_normal(n).astype(np.float32).view(np.uint32)
    elif kind == "signed0":
        v = rng.integers(-2, 3, n).astype(np.float32)
        v[rng.random(n) < 0.3] = -0.0
        v[rng.random(n) < 0.01] = np.inf
        v[rng.random(n) < 0.01] = -np.inf
        b = v.view(np.uint32)
    else:
        raise ValueError(kind)
    if dt == "f32" and kind not in ("normal", "signed0"):
        e = (b >> 23) & 0xFF
        b = np.where(e == 0xFF, b & ~np.uint32(1 << 30), b).astype(np.uint32)
    return np.ascontiguousarray(b, dtype=np.uint32)


def check_select(bits, dt, k, smallest):
    x = to_dev(bits, dt)
    ok, oi, ot = drtopk.drtopk_select(x, k, smallest=smallest, want_kth=True, dtype=dt)
    torch.cuda.synchronize()
    if smallest:
        rk, ri = oracle.bottomk(bits, DT[dt], k)
        rkth = oracle.kth_smallest(bits, DT[dt], k)
    else:
        rk, ri = oracle.topk(bits, DT[dt], k)
        rkth = oracle.kth(bits, DT[dt], k)
    gk, gi = host_bits(ok), oi.cpu().numpy()
    bad = np.nonzero((gk != rk) | (gi != ri))[0]
    assert bad.size == 0, "n=%d k=%d smallest=%s first mismatch %d: (%x,%d) vs (%x,%d)" % (
        bits.size, k, smallest, bad[0], gk[bad[0]], gi[bad[0]], rk[bad[0]], ri[bad[0]])
    assert int(host_bits(ot)[0]) == rkth
    # k-selection alone
    _, _, kt = drtopk.drtopk_select(x, k, smallest=smallest, want_topk=False, want_kth=True,
                                    dtype=dt)
    torch.cuda.synchronize()
    assert int(host_bits(kt)[0]) == rkth


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("kind", ["uniform", "few", "equal", "asc", "desc"])
def test_smallest_parity(dt, kind):
    for n in (1, 3, 100, 8193, 40000, 300007):
        bits = gen(kind, n, n + 1, dt)
        for k in sorted({1, min(n, 2), min(n, 100), max(1, n // 3), n}):
            check_select(bits, dt, k, smallest=True)


def test_smallest_float_specials_and_large_k():
    for n in (5000, 100003):
        for kind in ("signed0", "normal"):
            bits = gen(kind, n, 7, "f32")
            for k in (1, 17, n // 2, n):
                check_select(bits, "f32", k, smallest=True)
    n = 1 << 21
    for kind in ("uniform", "few", "asc"):
        bits = gen(kind, n, 9, "u32")
        for k in (4097, 65536, 300001):
            check_select(bits, "u32", k, smallest=True)
            check_select(bits, "u32", k, smallest=False)


def test_select_largest_equals_topk():
    bits = gen("few", 250007, 3, "i32")
    for k in (1, 999, 100000):
        check_select(bits, "i32", k, smallest=False)


def merge_case(bits, dt, cuts, k, smallest):
    """Shards [cuts[p], cuts[p+1]) of one device array, each through
    drtopk_select, merged; returns the merged (keys, int64 global idx)."""
    x = to_dev(bits, dt)
    lk, li, offs = [], [], [0]
    for a, b in zip(cuts[:-1], cuts[1:]):
        kk = min(k, b - a)
        ok, oi, _ = drtopk.drtopk_select(x[a:b], kk, smallest=smallest, dtype=dt)
        lk.append(ok)
        li.append(oi)
        offs.append(offs[-1] + kk)
    kc, ic = torch.cat(lk), torch.cat(li)
    kk = min(k, offs[-1])
    mk, mg = drtopk.drtopk_topk_merge(kc, ic, offs, cuts[:-1], kk, smallest=smallest, dtype=dt)
    torch.cuda.synchronize()
    return host_bits(mk), mg.cpu().numpy(), kk


@pytest.mark.parametrize("smallest", [False, True])
def test_merge_of_shards_equals_whole(smallest):
    n = (1 << 22) + 333
    cuts = [0, 1, 1000, 1001, 700003, 2000000, 2000005, n]
    for dt, kind in (("u32", "few"), ("u32", "uniform"), ("f32", "normal"), ("i32", "equal"),
                     ("u32", "asc")):
        bits = gen(kind, n, 21, dt)
        pick = oracle.bottomk if smallest else oracle.topk
        for k in (1, 5, 1000, 70000, 1 << 20):
            gk, gg, kk = merge_case(bits, dt, cuts, k, smallest)
            rk, ri = pick(bits, DT[dt], kk)
            assert np.array_equal(gk, rk) and np.array_equal(gg, ri.astype(np.int64)), \
                (dt, kind, k, smallest)


def test_merge_with_large_global_bases():
    """Eight sub-vectors of a vector longer than 2^31 keys: shard p is a
    separate array whose global base is p * 3 * 2^30; the merged indices
    must equal the oracle's merge of the oracle's shard lists."""
    P, m, k = 8, 300001, 50000
    lk, li, offs, ek, eg = [], [], [0], [], []
    bases = [p * 3 * (1 << 30) for p in range(P)]
    for p in range(P):
        bits = inputs.distinct16_u32(m, 30 + (p % 2)).numpy().view(np.uint32)
        ok, oi, _ = drtopk.drtopk_select(to_dev(bits, "u32"), k, dtype="u32")
        lk.append(ok)
        li.append(oi)
        offs.append(offs[-1] + k)
        rk, ri = oracle.topk(bits, oracle.U32, k)
        ek.append(rk)
        eg.append(ri.astype(np.int64) + bases[p])
    mk, mg = drtopk.drtopk_topk_merge(torch.cat(lk), torch.cat(li), offs, bases, k, dtype="u32")
    torch.cuda.synchronize()
    rk, rg = oracle.topk_merge(np.concatenate(ek), np.concatenate(eg), oracle.U32, k)
    assert np.array_equal(host_bits(mk), rk) and np.array_equal(mg.cpu().numpy(), rg)
    assert int(mg.max()) > 2**31


def test_merge_argument_checks():
    x = torch.zeros(10, dtype=torch.int32, device="cuda")
    i = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(drtopk.DrTopkError) as e:
        drtopk.drtopk_topk_merge(x, i, [0, 5, 10], [0, 100], 11, dtype="u32")
    assert e.value.status == 2
    with pytest.raises(drtopk.DrTopkError):
        drtopk.drtopk_topk_merge(x, i, [0, 6, 5], [0, 100], 3, dtype="u32")
