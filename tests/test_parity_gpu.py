"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Keys and indices must be bit-exact for every dtype, distribution, size and
k: the method is exact and ties go to the smallest index. Sizes span several
32 KB chunks and ragged tails; alpha and beta are also forced across their
whole range. Intermediate stages (delegates, threshold, |{x > tau}|) are
compared with the oracle's steps of Rules 1-3.
"""

import json
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_example.json")
DT = {"u32": oracle.U32, "i32": oracle.I32, "f32": oracle.F32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def to_dev(bits, dt):
    t = torch.from_numpy(np.ascontiguousarray(bits).view(np.int32).copy())
    if dt == "f32":
        t = t.view(torch.float32)
    return t.cuda()


def host_bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def make(kind, n, seed, dt):
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
    elif kind == "zero":
        b = np.zeros(n, np.uint32)
    elif kind == "normal":
        b = rng.standard_normal(n).astype(np.float32).view(np.uint32)
    elif kind == "zipf":
        b = inputs.zipf_u32(n, seed).numpy().view(np.uint32)
    elif kind == "signed0":
        v = rng.integers(-2, 3, n).astype(np.float32)
        v[rng.random(n) < 0.3] = -0.0
        b = v.view(np.uint32)
    else:
        raise ValueError(kind)
    if dt == "f32" and kind in ("uniform", "few", "asc", "desc", "equal", "zero", "zipf"):
        # keep f32 bit patterns finite: clear the top exponent bit pattern 0xFF
        e = (b >> 23) & 0xFF
        b = np.where(e == 0xFF, b & ~np.uint32(1 << 30), b).astype(np.uint32)
    return b


def check_topk(bits, dt, k, alpha=0, beta=0):
    x = to_dev(bits, dt)
    ok, oi, ot, st = drtopk.drtopk_topk_ex(x, k, alpha=alpha, beta=beta, dtype=dt)
    torch.cuda.synchronize()
    rk, ri = oracle.topk(bits, DT[dt], k)
    gk = host_bits(ok)
    gi = oi.cpu().numpy()
    assert st["error"] == 0, st
    assert st["emitted"] == k, st
    bad = np.nonzero((gk != rk) | (gi != ri))[0]
    assert bad.size == 0, "first mismatch at %d: gpu (%x,%d) oracle (%x,%d) stats %s" % (
        bad[0], gk[bad[0]], gi[bad[0]], rk[bad[0]], ri[bad[0]], st)
    assert int(host_bits(ot)[0]) == oracle.kth(bits, DT[dt], k)
    return st


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("kind", ["uniform", "few", "equal", "asc", "desc", "zipf"])
def test_topk_parity_sizes(dt, kind):
    for n in (1, 2, 3, 31, 100, 1000, 8191, 8192, 8193, 40000, 300007):
        bits = make(kind, n, n, dt)
        for k in sorted({1, 2, 7, min(n, 100), max(1, n // 3), n}):
            if k <= n:
                check_topk(bits, dt, k)


def test_topk_parity_float_specials():
    for n in (50, 5000, 100003):
        bits = make("signed0", n, 3, "f32")
        for k in (1, 10, n // 2, n):
            check_topk(bits, "f32", k)
        bits = make("normal", n, 4, "f32")
        for k in (1, 33, n // 7):
            check_topk(bits, "f32", k)


@pytest.mark.parametrize("beta", [1, 2, 3, 4])
def test_topk_parity_forced_alpha_beta(beta):
    n = 200003
    for kind in ("uniform", "few", "asc", "equal"):
        bits = make(kind, n, 11 + beta, "u32")
        for alpha in range(2, 17):
            for k in (1, 5, 300, 4097):
                check_topk(bits, "u32", k, alpha=alpha, beta=beta)


def test_kth_only_parity():
    for dt in ("u32", "i32", "f32"):
        for kind in ("uniform", "few", "equal", "desc"):
            n = 123457
            bits = make(kind, n, 5, dt)
            x = to_dev(bits, dt)
            for k in (1, 64, 5000, n):
                got = drtopk.drtopk_kth(x, k, dtype=dt)
                torch.cuda.synchronize()
                assert int(host_bits(got)[0]) == oracle.kth(bits, DT[dt], k), (dt, kind, k)


def test_large_k_sort_path():
    # k > 4096 uses the multi-block radix sort of the outputs
    n = 1 << 20
    for kind in ("uniform", "few", "asc", "zipf"):
        bits = make(kind, n, 21, "u32")
        for k in (4097, 65536, 300000):
            check_topk(bits, "u32", k)


@pytest.mark.parametrize("dt", ["u32", "f32"])
def test_delegates_match_oracle(dt):
    for kind in ("uniform", "few", "equal", "zero"):
        for n in (5, 1000, 8192 * 3 + 17, 100000):
            bits = make(kind, n, 7, dt)
            mapped = oracle.map_keys(bits, DT[dt])
            x = to_dev(bits, dt)
            for alpha in (2, 3, 4, 5, 6, 8, 11, 13, 14, 16):
                for beta in (1, 2, 3, 4):
                    dk, di = drtopk.drtopk_delegates(x, alpha, beta, dtype=dt)
                    torch.cuda.synchronize()
                    rk, ri = oracle.delegates(mapped, alpha, beta)
                    gk = dk.cpu().numpy().view(np.uint32)
                    gi = di.cpu().numpy().astype(np.int64)
                    assert np.array_equal(gk, rk), (kind, n, alpha, beta)
                    assert np.array_equal(gi, ri), (kind, n, alpha, beta)


def test_threshold_and_filter_counts_match_oracle_steps():
    for kind in ("uniform", "few", "asc", "zipf"):
        n = 1 << 18
        bits = make(kind, n, 9, "u32")
        mapped = oracle.map_keys(bits, oracle.U32)
        for alpha, beta, k in [(8, 2, 128), (5, 1, 1000), (10, 3, 17), (4, 4, 20000)]:
            st = check_topk(bits, "u32", k, alpha=alpha, beta=beta)
            dk, di = oracle.delegates(mapped, alpha, beta)
            tau = oracle.threshold(dk, di, k)
            assert st["tau"] == tau
            assert st["greater"] == int((mapped > tau).sum())
            if st["greater"] < k:
                assert st["ties_needed"] == k - st["greater"]


def test_paper_worked_example_on_gpu():
    g = json.load(open(GOLDEN))
    v = np.array(g["V"], np.uint32)
    x = to_dev(v, "u32")
    dk, di = drtopk.drtopk_delegates(x, g["alpha"], 1, dtype="u32")
    assert dk.cpu().numpy().view(np.uint32)[:, 0].tolist() == g["D_beta1"]
    for c in g["cases"]:
        ok, oi, ot, st = drtopk.drtopk_topk_ex(x, c["k"], alpha=g["alpha"], beta=c["beta"],
                                               dtype="u32")
        assert st["tau"] == c["tau"]
        assert host_bits(ok).tolist() == c["topk"]
        # the kept candidates >= tau are the paper's concatenated vector
        assert st["greater"] + st["ties_needed"] <= len(c["candidates"])
        assert st["greater"] == sum(1 for y in c["candidates"] if y > c["tau"])


def test_generated_workload_recipes_small():
    dev = torch.device("cuda")
    for name in inputs.ADVERSARIAL + ["uniform", "nd"]:
        x = inputs.DISTRIBUTIONS[name](1 << 16, 3, device=dev)
        bits = host_bits(x)
        for k in (1, 1024, 30000):
            check_topk(bits, "u32", k)
        # the same generator on the CPU gives the same bytes
        if name != "nd":
            assert np.array_equal(bits, host_bits(inputs.DISTRIBUTIONS[name](1 << 16, 3)))


def test_host_entry_point():
    """Host keys through the library's staging buffer: repeated shapes with
    new contents (graph replays), a larger call that grows the buffer, and
    the small shape again inside the grown buffer."""
    calls = [("few", 77777, 500, 1), ("uniform", 77777, 500, 2), ("asc", 77777, 500, 3),
             ("uniform", 300007, 70000, 4), ("few", 77777, 500, 5), ("zipf", 77777, 500, 6)]
    for kind, n, k, seed in calls:
        bits = make(kind, n, seed, "u32")
        ok, oi = drtopk.drtopk_topk_host(bits, k, "u32")
        rk, ri = oracle.topk(bits, oracle.U32, k)
        assert np.array_equal(ok, rk) and np.array_equal(oi, ri), (kind, n, k)


def test_streams_and_repeat_calls_are_independent():
    s = torch.cuda.Stream()
    bits = make("uniform", 1 << 17, 2, "u32")
    x = to_dev(bits, "u32")
    rk, ri = oracle.topk(bits, oracle.U32, 999)
    with torch.cuda.stream(s):
        outs = [drtopk.drtopk_topk(x, 999, dtype="u32", stream=s) for _ in range(4)]
    s.synchronize()
    for ok, oi in outs:
        assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)


def test_repeated_calls_see_new_data():
    """Identical arguments replay a cached graph of the query: each call must
    still read the current contents of the buffers."""
    n, k = 300001, 777
    x = torch.empty(n, dtype=torch.int32, device="cuda")
    ok = torch.empty(k, dtype=torch.int32, device="cuda")
    oi = torch.empty(k, dtype=torch.int32, device="cuda")
    kt = torch.empty(1, dtype=torch.int32, device="cuda")
    for it, kind in enumerate(["uniform", "few", "equal", "asc", "uniform"]):
        bits = make(kind, n, 40 + it, "u32")
        x.copy_(torch.from_numpy(bits.view(np.int32)))
        drtopk.drtopk_topk(x, k, out_keys=ok, out_idx=oi, dtype="u32")
        drtopk.drtopk_kth(x, k, out=kt, dtype="u32")
        torch.cuda.synchronize()
        rk, ri = oracle.topk(bits, oracle.U32, k)
        assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri), kind
        assert int(host_bits(kt)[0]) == int(rk[-1])


def test_many_distinct_calls_evict_cleanly():
    # more distinct argument sets than the graph cache keeps
    bits = make("uniform", 50000, 9, "u32")
    x = to_dev(bits, "u32")
    for k in range(1, 140):
        ok, oi = drtopk.drtopk_topk(x, k, dtype="u32")
        if k % 23 == 0:
            torch.cuda.synchronize()
            rk, ri = oracle.topk(bits, oracle.U32, k)
            assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)
    torch.cuda.synchronize()


def test_queries_inside_a_user_graph():
    """Calls on a stream under capture launch kernel by kernel into the
    caller's graph (workspace as graph allocation nodes)."""
    n, k = 200003, 513
    x = torch.empty(n, dtype=torch.int32, device="cuda")
    ok = torch.empty(k, dtype=torch.int32, device="cuda")
    oi = torch.empty(k, dtype=torch.int32, device="cuda")
    kt = torch.empty(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        drtopk.drtopk_topk(x, k, out_keys=ok, out_idx=oi, dtype="u32", stream=s)
        drtopk.drtopk_kth(x, 7, out=kt, dtype="u32", stream=s)
    for it, kind in enumerate(["uniform", "few", "desc"]):
        bits = make(kind, n, 70 + it, "u32")
        x.copy_(torch.from_numpy(bits.view(np.int32)))
        g.replay()
        torch.cuda.synchronize()
        rk, ri = oracle.topk(bits, oracle.U32, k)
        assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri), kind
        assert int(host_bits(kt)[0]) == oracle.kth(bits, oracle.U32, 7)


@pytest.mark.parametrize("flags", [(True, False), (False, True), (True, True)])
def test_ablations_stay_exact(flags):
    """Rule 2 off and / or the first select stopped one digit early change
    the candidate set, never the answer (Sec. 5 ablations)."""
    no_filter, skip_last = flags
    for kind in ("uniform", "few", "equal", "asc", "zipf", "normal"):
        n = 200003
        dt = "f32" if kind == "normal" else "u32"
        bits = make(kind, n, 31, dt)
        x = to_dev(bits, dt)
        for beta in (1, 2):
            for k in (1, 100, 5000, 70000):
                ok, oi, st = drtopk.drtopk_topk_ablate(x, k, beta=beta, no_filter=no_filter,
                                                       skip_last_digit=skip_last, dtype=dt)
                _, _, _, base = drtopk.drtopk_topk_ex(x, k, beta=beta, dtype=dt)
                rk, ri = oracle.topk(bits, DT[dt], k)
                assert st["error"] == 0, st
                assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri), \
                    (kind, beta, k, flags)
                if skip_last:
                    assert st["tau"] <= base["tau"] and (st["tau"] & 0xFF) == 0 or st["tau"] == 0
                if no_filter and not skip_last:
                    assert st["greater"] >= base["greater"]  # whole subranges kept


def test_tie_paths_dense_and_sparse():
    """Ties at tau over many tiles: sparse (ND-like, ties spread thinly; one
    tie needed among distinct keys) and dense (few values, all equal), with
    the cut falling inside the walk; checked against the oracle."""
    n = 1 << 22
    dev = torch.device("cuda")
    cases = [("nd", inputs.nd_u32(n, 5, device=dev), (1000, 65536, 500000)),
             ("distinct16", inputs.distinct16_u32(n, 6, device=dev), (1024, 300000, 1 << 20)),
             ("all_equal", inputs.all_equal_u32(n, device=dev), (7, 4096, 1 << 20)),
             ("uniform", inputs.uniform_u32(n, 7, device=dev), (1, 1024, 100000))]
    for name, x, ks in cases:
        bits = host_bits(x)
        for k in ks:
            for alpha in (0, 5, 9, 14):
                ok, oi, _, st = drtopk.drtopk_topk_ex(x, k, alpha=alpha, dtype="u32")
                rk, ri = oracle.topk(bits, oracle.U32, k)
                assert st["error"] == 0, (name, k, alpha, st)
                assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri), \
                    (name, k, alpha, st)


def test_large_scan_sets():
    """Scan sets of more than 2^22 keys (sorted input, large k: Rule 2 keeps
    k / beta whole subranges): select mode over many scan steps,
    k-selection, and tie mode with every subrange scanned."""
    n = 1 << 25
    large = 0
    for dt, kind in (("u32", "asc"), ("u32", "desc"), ("f32", "asc")):
        bits = make(kind, n, 41, dt)
        x = to_dev(bits, dt)
        mapped = oracle.map_keys(bits, DT[dt])
        for k, alpha in ((1 << 20, 0), (1 << 18, 6), (300001, 8)):
            st = check_topk(bits, dt, k, alpha=alpha)
            large += (st["scanned"] << st["alpha"]) > (1 << 22)
            assert st["greater"] >= k, st
            # |{x > tau}| stays exact when the scan set is counted first
            assert st["greater"] == int((mapped > st["tau"]).sum()), st
        got = drtopk.drtopk_kth(x, 1 << 20, dtype=dt)
        torch.cuda.synchronize()
        assert int(host_bits(got)[0]) == oracle.kth(bits, DT[dt], 1 << 20), (dt, kind)
    assert large >= 6
    # two large keys per 64-key subrange, zeros elsewhere: with k just above
    # the number of large keys, tau = 0, every subrange is scanned and the
    # last 1000 answers are the zeros of smallest index
    rng = np.random.default_rng(43)
    S = n >> 6
    bits = np.zeros(n, np.uint32)
    off = np.argsort(rng.random((S, 64)), axis=1)[:, :2]
    pos = (np.arange(S)[:, None] * 64 + off).ravel()
    bits[pos] = rng.integers(1, 2**32, pos.size, dtype=np.uint64).astype(np.uint32)
    k = 2 * S + 1000
    st = check_topk(bits, "u32", k, alpha=6, beta=2)
    assert st["tau"] == 0 and st["greater"] == 2 * S and st["ties_needed"] == 1000, st
    assert (st["scanned"] << 6) > (1 << 22), st
    got = drtopk.drtopk_kth(to_dev(bits, "u32"), k, dtype="u32")
    torch.cuda.synchronize()
    assert int(host_bits(got)[0]) == 0


def test_output_sort_clustered_winners():
    """Winners that share their high bits: many copies of the largest keys
    packed into a few subranges (so few delegates see them and the query
    stays in select mode). The output sort's buckets then hold more entries
    than one CTA sorts in shared memory, which takes its chunked merge path;
    the result must still equal the oracle's."""
    rng = np.random.default_rng(91)
    n = 1 << 22
    for copies, k, spread in ((20000, 30000, False), (70000, 100000, False),
                              (9000, 50000, True), (300000, 400000, False)):
        bits = rng.integers(0, 0xF0000000, n, dtype=np.uint64).astype(np.uint32)
        if spread:  # a few clusters of two top values
            for c0 in (1000, 2000000, 3000000):
                bits[c0:c0 + copies] = 0xFFFFFFF0
                bits[c0 + copies:c0 + 2 * copies] = 0xFFFFFFE0
        else:
            bits[5000:5000 + copies] = 0xFFFFFFF0
        st = check_topk(bits, "u32", k)
        assert st["greater"] >= k, st  # select mode: the sort covers all k
        check_topk(bits, "u32", k, alpha=4, beta=1)


def test_host_entry_point_in_pieces():
    """Host keys longer than one copy piece (32M keys): the delegate pass
    runs piece by piece as the copies land; ragged last piece, tie-heavy and
    distinct inputs, small and large k."""
    n = (1 << 26) + 3 * (1 << 20) + 12345
    for kind, ks in (("few", (1000, 300000)), ("uniform", (1, 1 << 20)), ("asc", (4096,))):
        bits = make(kind, n, 77, "u32")
        for k in ks:
            ok, oi = drtopk.drtopk_topk_host(bits, k, "u32")
            rk, ri = oracle.topk(bits, oracle.U32, k)
            assert np.array_equal(ok, rk) and np.array_equal(oi, ri), (kind, k)
