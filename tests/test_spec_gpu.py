"""Speculative compaction of the delegate vector (large arrays, alpha in
[5, 10]): a sample of the chunks bounds tau from below, the delegate pass
stores only the records of subranges whose largest delegate reaches that
bound, and the threshold and the classification read the records. Every
path is compared with the CPU oracle element by element at n = 2^26
(alpha = 6 at k = 2^16 by Rule 4), and the statistics say which path ran
(bit 0: records stored, bit 1: a fallback pass wrote the full delegate
arrays; after a declined sample that pass is the query's delegate pass):
  * records used and sufficient: uniform, sorted, Zipf, i32, the smallest
    criterion, k-selection alone (normal f32: records, or a declined sample);
  * the sample declines (every sampled delegate equal): the fallback pass
    writes the full arrays and takes the first-digit histogram;
  * the sample misleads (large keys only in the sampled chunks, more
    needed than they hold): tau < the bound, the full arrays are written
    and the query is still exact;
  * tie mode with records (the k-th key duplicated): the full arrays are
    written before the tie path reads them;
  * an unaligned base: not eligible (full arrays from the start).
"""

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 1 << 26
K = 1 << 16
CHUNK = 8192        # keys per chunk of the delegate pass
SAMPLE_STRIDE = 128  # every 128th chunk is sampled
DT = {"u32": oracle.U32, "i32": oracle.I32, "f32": oracle.F32}
TDT = {"u32": torch.int32, "i32": torch.int32, "f32": torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def host_bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def to_dev(bits, dt):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int32)).view(TDT[dt]).cuda()


def check(bits, dt, k, path, smallest=False, x=None):
    """Runs top-k (and the k-th) through drtopk_topk_ex or drtopk_select
    and compares with the oracle; returns the delegate path bits."""
    if x is None:
        x = to_dev(bits, dt)
    if smallest:
        ok, oi, ot = drtopk.drtopk_select(x, k, smallest=True, want_kth=True, dtype=dt)
        torch.cuda.synchronize()
        rk, ri = oracle.bottomk(bits, DT[dt], k)
        rkth = oracle.kth_smallest(bits, DT[dt], k)
        st = None
    else:
        assert drtopk.drtopk_plan(bits.size, k)[0] == 6
        ok, oi, ot, st = drtopk.drtopk_topk_ex(x, k, dtype=dt)
        rk, ri = oracle.topk(bits, DT[dt], k)
        rkth = oracle.kth(bits, DT[dt], k)
    gk, gi = host_bits(ok), oi.cpu().numpy()
    bad = np.nonzero((gk != rk) | (gi != ri))[0]
    assert bad.size == 0, "first mismatch at %d" % bad[0]
    assert int(host_bits(ot)[0]) == rkth
    if st is not None:
        assert st["error"] == 0
        if path is not None:
            assert st["delegate_path"] in ((path,) if isinstance(path, int) else path), st
    return st


@pytest.mark.parametrize("kind", ["uniform", "ascending", "descending", "zipf"])
def test_records_used(kind):
    bits = inputs.DISTRIBUTIONS[kind](N, 11).numpy().view(np.uint32)
    check(bits, "u32", K, path=1)


def test_records_f32_i32_and_smallest():
    # float keys: the sampled 11-bit bins hold two mantissa bits, often too
    # coarse to bound the records; the sample may decline
    f = inputs.normal_f32(N, 12).numpy().view(np.uint32)
    check(f, "f32", K, path=(1, 2))
    check(f, "f32", K, path=None, smallest=True)
    i = inputs.uniform_u32(N, 13).numpy().view(np.uint32)
    check(i, "i32", K, path=1)
    check(i, "i32", 3 * K, path=None, smallest=True)


def test_kth_only_with_records():
    bits = inputs.uniform_u32(N, 14).numpy().view(np.uint32)
    x = to_dev(bits, "u32")
    _, _, ot, st = drtopk.drtopk_topk_ex(x, K, want_topk=False, dtype="u32")
    assert int(host_bits(ot)[0]) == oracle.kth(bits, oracle.U32, K)
    assert st["delegate_path"] == 1


def test_sample_declines_equal_keys():
    bits = np.full(N, 0x9E3779B9, np.uint32)
    check(bits, "u32", K, path=2)
    d16 = inputs.distinct16_u32(N, 19).numpy().view(np.uint32)
    check(d16, "u32", K, path=2)


def test_misleading_sample_falls_back():
    # small keys everywhere, large ones only in the sampled chunks: the
    # sampled chunks hold 2^26 / 8192 / 128 * 128 subranges * 2 = 16384
    # delegates, fewer than k, so tau lies below the sampled bound
    rng = np.random.default_rng(15)
    bits = rng.integers(0, 1 << 20, N, dtype=np.uint64).astype(np.uint32)
    for c in range(0, N // CHUNK, SAMPLE_STRIDE):
        bits[c * CHUNK:(c + 1) * CHUNK] = rng.integers(1 << 31, 1 << 32, CHUNK,
                                                       dtype=np.uint64).astype(np.uint32)
    check(bits, "u32", K, path=3)


def test_tie_mode_with_records_falls_back():
    # distinct keys (an odd multiplier is a bijection of u32), then the
    # k-th largest copied over three small keys: |{x > v}| = k - 1, the
    # query ends in tie mode and needs the smallest of the four v positions
    i = np.arange(N, dtype=np.uint64)
    bits = ((i * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    v = oracle.kth(bits, oracle.U32, K)
    small = np.nonzero(bits < np.uint32(1 << 24))[0]
    pos = np.random.default_rng(16).choice(small, 3, replace=False)
    bits[pos] = v
    st = check(bits, "u32", K, path=3)
    assert st["ties_needed"] >= 1


def test_unaligned_base_is_not_eligible():
    bits = inputs.uniform_u32(N + 1, 17).numpy().view(np.uint32)
    big = to_dev(bits, "u32")
    x = big[1:]
    sub = bits[1:].copy()
    ok, oi, ot, st = drtopk.drtopk_topk_ex(x, K, dtype="u32")
    rk, ri = oracle.topk(sub, oracle.U32, K)
    assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)
    assert st["delegate_path"] == 0


def test_graph_replay_with_records():
    # the cached-graph path (drtopk_topk) runs the same passes
    bits = inputs.zipf_u32(N, 18).numpy().view(np.uint32)
    x = to_dev(bits, "u32")
    rk, ri = oracle.topk(bits, oracle.U32, K)
    outs = (torch.empty(K, dtype=torch.int32, device="cuda"),
            torch.empty(K, dtype=torch.int32, device="cuda"))
    for _ in range(3):
        drtopk.drtopk_topk(x, K, out_keys=outs[0], out_idx=outs[1], dtype="u32")
        torch.cuda.synchronize()
        assert np.array_equal(host_bits(outs[0]), rk) and np.array_equal(outs[1].cpu().numpy(), ri)
    drtopk.sync_status()


@pytest.mark.parametrize("beta", [1, 3, 4])
def test_records_with_forced_beta(beta):
    # the records hold beta delegates each; results stay exact on uniform
    # keys whatever the path (records; records then the tie-mode fallback,
    # since 2^26 random u32 keys repeat and the k-th may be tied; or a
    # declined sample) and on the misleading sample, which must never end
    # with the records alone (declined when the sampled bins are crowded,
    # else the records pass finds fewer than k delegates above the bound)
    bits = inputs.uniform_u32(N, 20 + beta).numpy().view(np.uint32)
    x = to_dev(bits, "u32")
    ok, oi, ot, st = drtopk.drtopk_topk_ex(x, K, alpha=6, beta=beta, dtype="u32")
    rk, ri = oracle.topk(bits, oracle.U32, K)
    assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)
    assert int(host_bits(ot)[0]) == oracle.kth(bits, oracle.U32, K)
    assert st["error"] == 0 and st["beta"] == beta and st["delegate_path"] in (1, 2, 3)
    if beta == 3:
        rng = np.random.default_rng(21)
        m = rng.integers(0, 1 << 20, N, dtype=np.uint64).astype(np.uint32)
        for c in range(0, N // CHUNK, SAMPLE_STRIDE):
            m[c * CHUNK:(c + 1) * CHUNK] = rng.integers(1 << 31, 1 << 32, CHUNK,
                                                        dtype=np.uint64).astype(np.uint32)
        ok, oi, _, st = drtopk.drtopk_topk_ex(to_dev(m, "u32"), K, alpha=6, beta=3, dtype="u32")
        rk, ri = oracle.topk(m, oracle.U32, K)
        assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)
        assert st["error"] == 0 and st["delegate_path"] in (2, 3)
