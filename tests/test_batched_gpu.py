"""Parity of the batched ragged top-k (one persistent launch over many rows)
with the CPU oracle, row by row, keys and indices bit-exact.

Rows cover the direct path (n <= 4096) and the delegate path with every
alpha/beta, the three dtypes, tie-heavy and sorted inputs, float specials,
rows starting at any element (not 16-byte aligned), device-resident row
arrays, plan reuse inside a CUDA graph, the tuning table, and the full
ragged workload (4096 float32 rows of 2^U[10, 22] keys, k_r <= 1024) on
sampled rows plus whole-batch properties.
"""

import math

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu

DT = {"u32": oracle.U32, "i32": oracle.I32, "f32": oracle.F32}
KINDS = ["uniform", "few", "equal", "asc", "desc", "zero", "normal", "signed0"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def row_bits(kind, n, rng, dt):
    if kind == "uniform":
        b = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    elif kind == "few":
        b = rng.integers(0, 4, n).astype(np.uint32) * np.uint32(0x01010101)
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
    elif kind == "signed0":
        v = rng.integers(-2, 3, n).astype(np.float32)
        v[rng.random(n) < 0.3] = -0.0
        b = v.view(np.uint32)
    else:
        raise ValueError(kind)
    if dt == "f32":
        e = (b >> 23) & 0xFF
        b = np.where(e == 0xFF, b & ~np.uint32(1 << 30), b).astype(np.uint32)
    return b


def build_batch(lens, kinds, seed, dt, gap_max=3):
    """Concatenates rows with random gaps of 0..gap_max keys, so that row
    starts fall on any element."""
    rng = np.random.default_rng(seed)
    parts, off, pos = [], [], 0
    for n, kind in zip(lens, kinds):
        g = int(rng.integers(0, gap_max + 1))
        if g:
            parts.append(rng.integers(0, 2**32, g, dtype=np.uint64).astype(np.uint32))
            pos += g
        off.append(pos)
        parts.append(row_bits(kind, n, rng, dt))
        pos += n
    off.append(pos)
    return np.concatenate(parts), np.array(off, np.int64)


def to_dev(bits, dt):
    t = torch.from_numpy(np.ascontiguousarray(bits).view(np.int32).copy())
    if dt == "f32":
        t = t.view(torch.float32)
    return t.cuda()


def host_bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def run_and_check(bits, row_off, ks, dt, alpha=0, beta=0, rows_to_check=None):
    x = to_dev(bits, dt)
    plan = drtopk.BatchPlan(row_off, ks, dt, alpha=alpha, beta=beta)
    ok, oi = plan.run(x)
    plan.status()
    gk, gi = host_bits(ok), oi.cpu().numpy()
    check = range(len(ks)) if rows_to_check is None else rows_to_check
    for r in check:
        a, b = int(row_off[r]), int(row_off[r + 1])
        o0 = int(plan.out_off[r])
        rk, ri = oracle.topk(bits[a:b], DT[dt], int(ks[r]))
        sk, si = gk[o0:o0 + ks[r]], gi[o0:o0 + ks[r]]
        bad = np.nonzero((sk != rk) | (si != ri))[0]
        assert bad.size == 0, "row %d (n=%d k=%d) first mismatch at %d: (%x,%d) vs (%x,%d)" % (
            r, b - a, ks[r], bad[0], sk[bad[0]], si[bad[0]], rk[bad[0]], ri[bad[0]])
    params = plan.params()
    plan.close()
    return params


def loguniform_lengths(rng, rows, lo, hi):
    return [int(round(2.0 ** rng.uniform(lo, hi))) for _ in range(rows)]


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
def test_batched_ragged_mixed_rows(dt):
    rng = np.random.default_rng(100 + DT[dt])
    rows = 240
    lens = loguniform_lengths(rng, rows, 0, 18)
    lens[:6] = [1, 2, 4096, 4097, 8192, 8193]
    kinds = [KINDS[i % len(KINDS)] for i in range(rows)]
    ks = []
    for n in lens:
        c = int(rng.integers(0, 4))
        kmax = min(n, 4096)
        ks.append([1, kmax, int(rng.integers(1, kmax + 1)), min(kmax, 1024)][c])
    # rows are back to back but the first row starts at an odd element
    bits, _ = build_batch(lens, kinds, 7, dt, gap_max=0)
    bits = np.concatenate([np.array([5], np.uint32), bits])
    row_off = np.concatenate([[1], 1 + np.cumsum(lens)]).astype(np.int64)
    run_and_check(bits, row_off, np.array(ks, np.int32), dt)


@pytest.mark.parametrize("beta", [1, 2, 3, 4])
def test_batched_forced_alpha_beta(beta):
    rng = np.random.default_rng(beta)
    lens = [50001, 131072, 200003, 77777, 4097, 9000]
    kinds = ["uniform", "few", "asc", "equal", "desc", "normal"]
    bits, _ = build_batch(lens, kinds, beta, "u32", gap_max=0)
    row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    for alpha in [1] + list(range(5, 17)):
        for k in (1, 37, 1000, 4096):
            ks = np.array([min(k, n) for n in lens], np.int32)
            a, b = run_and_check(bits, row_off, ks, "u32", alpha=alpha, beta=beta)
            for n, ar, br in zip(lens, a, b):
                if alpha == 1:   # direct select where the row fits on chip
                    if n <= drtopk.batch_limits()["direct_max_onchip"]:
                        assert (ar, br) == (0, 0)
                    continue
                assert br == beta
                # raised only to keep beta * S on chip
                amin = 5
                while beta * math.ceil(n / 2**amin) > drtopk.batch_limits()["max_delegates"]:
                    amin += 1
                assert ar == max(alpha, amin)


def expected_params(n, k, lim):
    """The default per-row choice (no table entry)."""
    if n <= lim["direct_max"]:
        return 0, 0
    if n <= lim["direct_max_onchip"] and 2 * math.ceil(n / 32) < 2 * k:
        return 0, 0
    r4 = int(math.floor(0.5 * (math.log2(n) - math.log2(k) + 3)))
    amin = 5
    while 2 * math.ceil(n / 2**amin) > lim["max_delegates"]:
        amin += 1
    a = min(max(r4, amin), 16)
    while a > amin and 2 * math.ceil(n / 2**a) < 2 * k:
        a -= 1
    return a, 2


def test_batched_parameters_follow_rule4_and_table():
    lim = drtopk.batch_limits()
    lens = [100, 4096, 4097, 10000, 40000, 1 << 16, 1 << 20, (1 << 22) + 3, 16500]
    ks = [7, 4096, 5, 700, 4000, 1024, 1000, 1, 600]
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2**32, sum(lens), dtype=np.uint64).astype(np.uint32)
    row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    a, b = run_and_check(bits, row_off, np.array(ks, np.int32), "u32")
    for n, k, ar, br in zip(lens, ks, a, b):
        assert (ar, br) == expected_params(n, k, lim), (n, k, ar, br)
    assert a[3] == 0 and a[4] > 0   # 10000/700 is selected directly, 40000 is too long
    # table entries override the default for their shape bucket
    drtopk.tune_set(20, 9, 12, 3)   # n in [2^20, 2^21), k in [512, 1024)
    drtopk.tune_set(14, 9, 6, 4)    # n in [2^14, 2^15), k in [512, 1024): delegates
    try:
        a, b = run_and_check(bits, row_off, np.array(ks, np.int32), "u32")
        assert (a[6], b[6]) == (12, 3)
        assert (a[5], b[5]) == expected_params(lens[5], ks[5], lim)
        assert (a[8], b[8]) == (6, 4)
        drtopk.tune_set(20, 9, 1, 0)  # direct, but 2^20 keys do not fit on chip
        a, b = run_and_check(bits, row_off, np.array(ks, np.int32), "u32")
        assert (a[6], b[6]) == expected_params(lens[6], ks[6], lim)
    finally:
        drtopk.tune_set(20, 9, 0, 0)
        drtopk.tune_set(14, 9, 0, 0)


def test_batched_unaligned_starts_and_gaps():
    """Rows that start at every residue mod 4 keys and sit between unused keys."""
    rng = np.random.default_rng(11)
    lens, kinds, starts = [], [], []
    parts, pos = [], 0
    for r in range(64):
        g = r % 4 + 4 * int(rng.integers(0, 3))
        parts.append(rng.integers(0, 2**32, g, dtype=np.uint64).astype(np.uint32))
        pos += g
        n = int(rng.integers(1, 70000))
        starts.append(pos)
        parts.append(row_bits(KINDS[r % 6], n, rng, "u32"))
        pos += n
        lens.append(n)
    bits = np.concatenate(parts)
    x = to_dev(bits, "u32")
    # one plan per row set: rows must be contiguous, so a gap is a row of its own
    off = []
    ks = []
    is_row = []
    cur = 0
    for s, n in zip(starts, lens):
        if s > cur:
            off.append(cur)
            ks.append(1)
            is_row.append(False)
        off.append(s)
        ks.append(int(min(n, rng.integers(1, 3000))))
        is_row.append(True)
        cur = s + n
    off.append(cur)
    off = np.array(off, np.int64)
    ks = np.array(ks, np.int32)
    check = [i for i, f in enumerate(is_row) if f]
    run_and_check(bits, off, ks, "u32", rows_to_check=check)
    del x


def test_batched_plan_graph_replay_and_device_row_arrays():
    rng = np.random.default_rng(5)
    lens = loguniform_lengths(rng, 100, 8, 17)
    ks = np.array([int(rng.integers(1, min(n, 1024) + 1)) for n in lens], np.int32)
    row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(row_off[-1])
    x = torch.empty(total, dtype=torch.float32, device="cuda")
    plan = drtopk.BatchPlan(row_off, ks, "f32")
    ok = torch.empty(plan.total_k, dtype=torch.float32, device="cuda")
    oi = torch.empty(plan.total_k, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(x, ok, oi, stream=s)  # warm-up outside capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(x, ok, oi, stream=s)
    for it in range(3):
        bits = rng.standard_normal(total).astype(np.float32).view(np.uint32)
        x.copy_(torch.from_numpy(bits.view(np.float32)))
        g.replay()
        torch.cuda.synchronize()
        plan.status()
        gk, gi = host_bits(ok), oi.cpu().numpy()
        for r in range(len(lens)):
            a, b = row_off[r], row_off[r + 1]
            o0 = plan.out_off[r]
            rk, ri = oracle.topk(bits[a:b], oracle.F32, int(ks[r]))
            assert np.array_equal(gk[o0:o0 + ks[r]], rk) and np.array_equal(
                gi[o0:o0 + ks[r]], ri), (it, r)
    plan.close()
    # the one-shot entry with row arrays in device memory
    d_off = torch.from_numpy(row_off).cuda()
    d_ks = torch.from_numpy(ks).cuda()
    L = drtopk.lib()
    import ctypes
    ok2 = torch.empty(int(ks.sum()), dtype=torch.float32, device="cuda")
    oi2 = torch.empty(int(ks.sum()), dtype=torch.int32, device="cuda")
    rc = L.drtopk_topk_batched(ctypes.c_void_p(x.data_ptr()), drtopk.F32,
                               ctypes.cast(d_off.data_ptr(), ctypes.POINTER(ctypes.c_int64)),
                               ctypes.cast(d_ks.data_ptr(), ctypes.POINTER(ctypes.c_int32)),
                               len(lens), ctypes.c_void_p(ok2.data_ptr()),
                               ctypes.c_void_p(oi2.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert torch.equal(ok2.view(torch.int32), ok.view(torch.int32))
    assert torch.equal(oi2, oi)


def ordered(f):
    """float32 tensor -> int64 keys in the library's total order (-0.0 below
    +0.0), computed from the bits with plain torch integer ops."""
    b = f.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    return torch.where(b >= (1 << 31), 0xFFFFFFFF - b, b + (1 << 31))


def test_batched_full_ragged_workload():
    """4096 float32 rows, lengths round(2^U[10, 22]), k_r uniform in
    [1, min(1024, n_r)], keys N(0, 1): the oracle on 160 rows (the 32 longest
    and 128 others) and, on every row, exact-answer properties."""
    lens, ks = inputs.batched_rows(4096, 4)
    row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(row_off[-1])
    x = inputs.normal_f32(total, 4, device=torch.device("cuda"))
    ks = np.array(ks, np.int32)
    plan = drtopk.BatchPlan(row_off, ks, "f32")
    ok, oi = plan.run(x)
    plan.status()
    # every row: indices in range, keys read back at them, sorted by
    # (key desc, index asc)
    out_off = torch.from_numpy(plan.out_off).cuda()
    row_of = torch.repeat_interleave(torch.arange(4096, device="cuda"),
                                     torch.from_numpy(ks.astype(np.int64)).cuda())
    starts = torch.from_numpy(row_off[:-1]).cuda()[row_of]
    lens_t = torch.from_numpy(np.array(lens, np.int64)).cuda()[row_of]
    idx = oi.to(torch.int64)
    assert bool(((idx >= 0) & (idx < lens_t)).all())
    assert torch.equal(x[starts + idx], ok)
    same_row = row_of[1:] == row_of[:-1]
    kd = ok[1:] - ok[:-1]
    assert bool((~same_row | (kd <= 0)).all())
    tie = same_row & (ok[1:] == ok[:-1])
    assert bool((~tie | (idx[1:] > idx[:-1])).all())
    # completeness, row by row: with kth_r the row's last output key, the
    # row holds exactly as many keys above kth_r as were returned above it,
    # and its keys equal to kth_r at indices up to the largest returned tie
    # index are exactly the returned ties (so the smallest indices won)
    ks_t = torch.from_numpy(ks.astype(np.int64)).cuda()
    last = out_off[1:] - 1
    kth_m = ordered(ok)[last]
    tmax = idx[last]
    out_gt = torch.zeros(4096, dtype=torch.int64, device="cuda")
    out_gt.scatter_add_(0, row_of, (ordered(ok) > kth_m[row_of]).to(torch.int64))
    in_gt = torch.zeros_like(out_gt)
    in_eq = torch.zeros_like(out_gt)
    r0 = 0
    while r0 < 4096:  # chunks of rows, about 2^26 keys each
        r1 = r0 + 1
        while r1 < 4096 and row_off[r1 + 1] - row_off[r0] <= (1 << 26):
            r1 += 1
        a, b = int(row_off[r0]), int(row_off[r1])
        seg = torch.repeat_interleave(torch.arange(r0, r1, device="cuda"),
                                      torch.from_numpy(np.diff(row_off[r0:r1 + 1])).cuda())
        m = ordered(x[a:b])
        pos = torch.arange(a, b, device="cuda") - torch.from_numpy(row_off).cuda()[seg]
        in_gt.scatter_add_(0, seg, (m > kth_m[seg]).to(torch.int64))
        in_eq.scatter_add_(0, seg, ((m == kth_m[seg]) & (pos <= tmax[seg])).to(torch.int64))
        r0 = r1
    assert torch.equal(in_gt, out_gt)
    assert torch.equal(in_eq, ks_t - out_gt)
    del out_off
    bits = None
    order = np.argsort(-np.array(lens))
    sample = sorted(set(order[:32].tolist()) |
                    set(np.random.default_rng(1).choice(4096, 128, replace=False).tolist()))
    gk, gi = host_bits(ok), oi.cpu().numpy()
    for r in sample:
        a, b = int(row_off[r]), int(row_off[r + 1])
        row = x[a:b].cpu().numpy().view(np.uint32)
        rk, ri = oracle.topk(row, oracle.F32, int(ks[r]))
        o0 = int(plan.out_off[r])
        assert np.array_equal(gk[o0:o0 + ks[r]], rk), r
        assert np.array_equal(gi[o0:o0 + ks[r]], ri), r
    plan.close()
    del x, bits
    torch.cuda.empty_cache()


def test_autotuned_table_stays_exact():
    """drtopk_autotune_batched measures (alpha, beta) per (log2 n, log2 k)
    bucket and fills the tuning table; plans built from that table must give
    the oracle's answer row by row. The table is restored afterwards."""
    lo, hi = 12, 16
    saved = {(ln, lk): drtopk.tune_get(ln, lk) for ln in range(lo, hi + 1) for lk in range(13)}
    try:
        drtopk.autotune_batched("f32", lo, hi, rows_per_shape=8)
        tuned = {key: drtopk.tune_get(*key) for key in saved}
        # every bucket the tuner covers (n > 4096, 2^lk <= min(4096, n / 2)) holds
        # a valid choice: the direct select or alpha in [5, 16] with beta in [1, 4]
        for (ln, lk), (a, b) in tuned.items():
            if ln > 12 and (1 << lk) <= min(4096, (1 << ln) // 2):
                assert a == 1 or (5 <= a <= 16 and 1 <= b <= 4), (ln, lk, a, b)
        rng = np.random.default_rng(23)
        lens, ks = [], []
        for ln in range(13, hi + 1):
            for lk in range(0, 13):
                if (1 << lk) > min(4096, (1 << ln) // 2):
                    continue
                for _ in range(2):
                    n = int(rng.integers(1 << ln, 1 << (ln + 1)))
                    lens.append(n)
                    ks.append(int(min(n, 4096, rng.integers(1 << lk, 1 << (lk + 1)))))
        row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        for kind in ("normal", "few"):
            bits = np.concatenate([row_bits(kind, n, rng, "f32") for n in lens])
            x = torch.from_numpy(bits.view(np.float32)).cuda()
            plan = drtopk.BatchPlan(row_off, ks, "f32")
            pa, pb = plan.params()
            used = {(int(a), int(b)) for a, b in zip(pa, pb)}
            ok, oi = plan.run(x)
            plan.status()
            gk, gi = host_bits(ok), oi.cpu().numpy()
            for r, n in enumerate(lens):
                a, b = int(row_off[r]), int(row_off[r + 1])
                rk, ri = oracle.topk(bits[a:b], oracle.F32, ks[r])
                o0 = int(plan.out_off[r])
                assert np.array_equal(gk[o0:o0 + ks[r]], rk), (kind, r, n, ks[r], pa[r], pb[r])
                assert np.array_equal(gi[o0:o0 + ks[r]], ri), (kind, r, n, ks[r], pa[r], pb[r])
            plan.close()
            assert len(used) > 1, used  # the table steered rows to different parameters
    finally:
        for (ln, lk), (a, b) in saved.items():
            drtopk.tune_set(ln, lk, a, b)
