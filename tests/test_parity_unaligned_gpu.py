"""Single queries on key arrays that start 4, 8 or 12 bytes past a 16-byte
boundary, against the CPU oracle element by element.

Such a base takes the plain-load variant of the delegate pass (bulk copies
need 16-byte aligned sources) and shifts the tie path's bulk copies to start
at the 16-byte block holding the first key. Sizes run from 1 key to above
2^22 keys, with sizes whose last 16-byte block is partial; inputs include
tie-heavy ones (all equal, 16 distinct values, ND-like) with k large enough
to reach the dense tie walk and the sparse tie path. The three entry points
drtopk_topk, drtopk_kth and drtopk_topk_ex are exercised (the first two
twice, so the second call replays a cached graph).
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
TORCH_DT = {"u32": torch.int32, "i32": torch.int32, "f32": torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def host_bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def gen(kind, n, seed, dt):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        b = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    elif kind == "equal":
        b = np.full(n, 0x9E3779B9, np.uint32)
    elif kind == "distinct16":
        vals = rng.integers(0, 2**32, 16, dtype=np.uint64).astype(np.uint32)
        b = vals[rng.integers(0, 16, n)]
    elif kind == "nd":
        b = inputs.nd_u32(n, seed).numpy().view(np.uint32)
    elif kind == "asc":
        b = (np.arange(n, dtype=np.uint64) * 4 + rng.integers(0, 4, n)).astype(np.uint32)
    elif kind == "normal":
        b = rng.standard_normal(n).astype(np.float32).view(np.uint32)
    else:
        raise ValueError(kind)
    if dt == "f32" and kind != "normal":
        e = (b >> 23) & 0xFF  # keep bit patterns finite
        b = np.where(e == 0xFF, b & ~np.uint32(1 << 30), b).astype(np.uint32)
    return np.ascontiguousarray(b, dtype=np.uint32)


def unaligned(bits, dt, off):
    """A device view of `bits` starting `off` elements past a 16-byte
    boundary (a slice of a larger allocation)."""
    n = bits.size
    buf = torch.empty(n + 8, dtype=TORCH_DT[dt], device="cuda")
    buf.view(torch.int32).fill_(0x5A5A5A5A)  # neighbours that must never be picked
    x = buf[off:off + n]
    x.view(torch.int32).copy_(torch.from_numpy(bits.view(np.int32)))
    assert x.data_ptr() % 16 == 4 * off
    return x, buf


def check(bits, dt, k, off, alpha=0, beta=0):
    x, _buf = unaligned(bits, dt, off)
    rk, ri = oracle.topk(bits, DT[dt], k)
    rkth = oracle.kth(bits, DT[dt], k)
    ok, oi, ot, st = drtopk.drtopk_topk_ex(x, k, alpha=alpha, beta=beta, dtype=dt)
    assert st["error"] == 0, st
    gk, gi = host_bits(ok), oi.cpu().numpy()
    bad = np.nonzero((gk != rk) | (gi != ri))[0]
    assert bad.size == 0, "n=%d k=%d off=%d first mismatch at %d: gpu (%x,%d) oracle (%x,%d) %s" % (
        bits.size, k, off, bad[0], gk[bad[0]], gi[bad[0]], rk[bad[0]], ri[bad[0]], st)
    assert int(host_bits(ot)[0]) == rkth
    if alpha or beta:
        return st
    for _ in range(2):  # plain entry points; the second call replays a graph
        ok2, oi2 = drtopk.drtopk_topk(x, k, dtype=dt)
        kt = drtopk.drtopk_kth(x, k, dtype=dt)
        torch.cuda.synchronize()
        assert np.array_equal(host_bits(ok2), rk) and np.array_equal(oi2.cpu().numpy(), ri)
        assert int(host_bits(kt)[0]) == rkth
    return st


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("off", [1, 2, 3])
def test_unaligned_sizes(dt, off):
    # sizes with every remainder mod 4 (a partial last 16-byte block), one
    # key, one 32 KB chunk and its neighbours, and several chunks
    for n in (1, 2, 3, 5, 6, 7, 33, 1001, 8190, 8191, 8192, 8193, 8194, 65537, 262147):
        for kind in ("uniform", "distinct16"):
            bits = gen(kind, n, n + off, dt)
            for k in sorted({1, min(n, 3), max(1, n // 5), n}):
                check(bits, dt, k, off)


@pytest.mark.parametrize("off", [1, 2, 3])
def test_unaligned_above_2p22_with_ties(off):
    """More than 2^22 keys, tie-heavy: the dense tie walk (all equal, 16
    distinct values) and the sparse tie path (ND-like) over many tiles."""
    n = (1 << 22) + 4093
    for kind, ks in (("equal", (5, 4096, 1 << 20)),
                     ("distinct16", (1024, 300001, 1 << 20)),
                     ("nd", (1000, 65536, 500000)),
                     ("uniform", (1, 1024, 100000)),
                     ("asc", (1 << 20,))):
        bits = gen(kind, n, 17 + off, "u32")
        for k in ks:
            check(bits, "u32", k, off)


def test_unaligned_forced_parameters_and_dtypes():
    """alpha below 5 (subranges inside one thread's keys), alpha above 13
    (subranges spanning chunks) and every beta, on i32 and f32 views."""
    n = 200003
    for dt, kind in (("i32", "distinct16"), ("f32", "normal"), ("u32", "equal")):
        bits = gen(kind, n, 5, dt)
        for alpha in (2, 4, 6, 11, 14, 16):
            for beta in (1, 2, 4):
                for k in (1, 777, 70001):
                    check(bits, dt, k, 1 + (alpha % 3), alpha=alpha, beta=beta)
