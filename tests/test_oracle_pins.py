"""Pins on the CPU oracle: it is checked against things other than itself.

* brute force (Python ``sorted`` over the typed values, IEEE total order for
  floats written out) on tiny inputs, every k;
* the paper's worked example (tests/golden/paper_example.json, cited there);
* special cases with known answers and the invariants of the definition;
* a library cross-check of values against ``torch.topk`` on distinct keys;
* the method equals the definition (Rules 1-3 lose nothing) for every alpha
  and beta on tie-heavy inputs;
* Rule 4's closed form against the paper's printed alpha(2^30, 2^24) = 4 and
  against a symbolic derivation from Eq. 6.
"""

import json
import math
import os
import struct

import numpy as np
import pytest
import torch

import oracle
from paper_2109_08219_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_example.json")


# ---------------------------------------------------------------- helpers ---

def _rng(seed):
    return np.random.default_rng(seed)


def small_input(rng, n, kind, dtype):
    """Tiny typed arrays with many ties and edge values."""
    if kind == "few":
        v = rng.integers(0, 4, n)
    elif kind == "equal":
        v = np.full(n, 7)
    elif kind == "asc":
        v = np.arange(n)
    elif kind == "desc":
        v = np.arange(n)[::-1]
    else:
        v = rng.integers(-1000, 1000, n)
    if dtype == np.float32:
        x = (v.astype(np.float64) - 1.5).astype(np.float32)
        if kind == "few" and n > 0:
            # plant signed zeros and infinities
            x[rng.integers(0, n, max(1, n // 5))] = -0.0
            x[rng.integers(0, n, max(1, n // 5))] = 0.0
            x[rng.integers(0, n, 1)] = np.float32(np.inf)
            x[rng.integers(0, n, 1)] = np.float32(-np.inf)
        return x
    if dtype == np.int32:
        return (v - 2).astype(np.int32)
    return (v.astype(np.int64) * 977 + (1 << 31)).astype(np.uint32) if kind == "rand" \
        else v.astype(np.uint32)


def brute_order(x):
    """Positions sorted by (value desc, index asc); -0.0 ranks below +0.0."""
    vals = x.tolist()
    if x.dtype == np.float32:
        def key(i):
            v = vals[i]
            negzero = 1 if (v == 0.0 and math.copysign(1.0, v) < 0) else 0
            return (-v, negzero, i)
    else:
        def key(i):
            return (-int(vals[i]), 0, i)
    return sorted(range(len(vals)), key=key)


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


# ------------------------------------------------------------- key map -------

def test_map_orders_floats_like_ieee_total_order():
    rng = _rng(0)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -1.0,
                         np.finfo(np.float32).max, -np.finfo(np.float32).max,
                         np.finfo(np.float32).tiny, -np.finfo(np.float32).tiny,
                         1e-45, -1e-45, 3.0, 3.0000002], dtype=np.float32)
    x = np.concatenate([specials, rng.standard_normal(150).astype(np.float32) * 1e3])
    bits, dt = oracle.as_bits(x)
    m = oracle.map_keys(bits, dt).astype(np.int64)
    xv = x.astype(np.float64)
    sb = np.signbit(x)
    less = (xv[:, None] < xv[None, :]) | (
        (xv[:, None] == 0) & (xv[None, :] == 0) & sb[:, None] & ~sb[None, :])
    equal_bits = bits[:, None] == bits[None, :]
    assert np.array_equal(m[:, None] < m[None, :], less)
    assert np.array_equal(m[:, None] == m[None, :], equal_bits)


def test_map_orders_i32_and_u32():
    rng = _rng(1)
    xi = np.concatenate([np.array([-2**31, 2**31 - 1, 0, -1, 1], np.int64),
                         rng.integers(-2**31, 2**31, 200)]).astype(np.int32)
    bits, dt = oracle.as_bits(xi)
    m = oracle.map_keys(bits, dt).astype(np.int64)
    a = xi.astype(np.int64)
    assert np.array_equal(m[:, None] < m[None, :], a[:, None] < a[None, :])
    xu = rng.integers(0, 2**32, 200, dtype=np.uint64).astype(np.uint32)
    bits, dt = oracle.as_bits(xu)
    assert np.array_equal(oracle.map_keys(bits, dt), xu)


def test_unmap_inverts_map():
    rng = _rng(2)
    raw = rng.integers(0, 2**32, 5000, dtype=np.uint64).astype(np.uint32)
    for dt in (oracle.U32, oracle.I32, oracle.F32):
        assert np.array_equal(oracle.unmap_keys(oracle.map_keys(raw, dt), dt), raw)


# --------------------------------------------------- plain definition -------

@pytest.mark.parametrize("dtype", [np.uint32, np.int32, np.float32])
@pytest.mark.parametrize("kind", ["few", "equal", "asc", "desc", "rand"])
def test_topk_matches_brute_force(dtype, kind):
    for seed in range(12):
        rng = _rng(100 + seed)
        n = int(rng.integers(1, 97))
        x = small_input(rng, n, kind, dtype)
        order = brute_order(x)
        bits, dt = oracle.as_bits(x)
        ks = range(1, n + 1) if n <= 40 else sorted({1, 2, n // 3, n // 2, n - 1, n})
        for k in ks:
            ok, oi = oracle.topk(bits, dt, k)
            assert oi.tolist() == order[:k], (n, k)
            assert np.array_equal(ok, bits[np.array(order[:k])])
            assert oracle.kth(bits, dt, k) == int(bits[order[k - 1]])


def test_topk_brute_force_larger():
    # n up to 4096, sampled k, tie-heavy and distinct inputs
    for seed, n in [(7, 1000), (8, 4096), (9, 2500)]:
        rng = _rng(seed)
        for x in (rng.integers(0, 16, n).astype(np.uint32),
                  rng.standard_normal(n).astype(np.float32),
                  rng.integers(-5, 5, n).astype(np.int32)):
            order = brute_order(x)
            bits, dt = oracle.as_bits(x)
            for k in (1, 5, 64, n // 2, n - 1, n):
                _, oi = oracle.topk(bits, dt, k)
                assert oi.tolist() == order[:k]


def test_special_cases():
    n = 300
    eq = np.full(n, 5, np.uint32)
    asc = np.arange(n, dtype=np.uint32)
    desc = asc[::-1].copy()
    for k in (1, 17, n):
        assert oracle.topk(eq, oracle.U32, k)[1].tolist() == list(range(k))
        assert oracle.topk(asc, oracle.U32, k)[1].tolist() == list(range(n - 1, n - 1 - k, -1))
        assert oracle.topk(desc, oracle.U32, k)[1].tolist() == list(range(k))
    rng = _rng(3)
    x = rng.integers(0, 50, n).astype(np.uint32)
    ok, oi = oracle.topk(x, oracle.U32, 1)
    assert ok[0] == x.max() and oi[0] == int(np.argmax(x))  # argmax = first max
    ok, oi = oracle.topk(x, oracle.U32, n)  # k = n: a full stable sort
    stable = np.argsort(-x.astype(np.int64), kind="stable")
    assert np.array_equal(oi, stable)


@pytest.mark.parametrize("dtype", [np.uint32, np.int32, np.float32])
def test_invariants(dtype):
    rng = _rng(4)
    for n in (1, 2, 33, 1000):
        x = small_input(rng, n, "few", dtype)
        bits, dt = oracle.as_bits(x)
        m = oracle.map_keys(bits, dt).astype(np.int64)
        for k in sorted({1, n // 2 or 1, n}):
            ok, oi = oracle.topk(bits, dt, k)
            kth = int(oracle.map_keys(np.array([oracle.kth(bits, dt, k)], np.uint32), dt)[0])
            mo = oracle.map_keys(ok, dt).astype(np.int64)
            assert len(ok) == k and len(set(oi.tolist())) == k
            assert oi.min() >= 0 and oi.max() < n
            assert np.array_equal(ok, bits[oi])
            assert (mo >= kth).all()
            assert int((m > kth).sum()) < k <= int((m >= kth).sum())
            assert (np.diff(mo) <= 0).all()
            tie = mo[1:] == mo[:-1]
            assert (np.diff(oi.astype(np.int64))[tie] > 0).all()


def test_values_match_torch_topk_on_distinct_keys():
    rng = _rng(5)
    x = rng.permutation(200000).astype(np.float32) * np.float32(0.37) - 1000
    bits, dt = oracle.as_bits(x)
    for k in (1, 10, 1000, 50000):
        ok, _ = oracle.topk(bits, dt, k)
        ref = torch.topk(torch.from_numpy(x), k).values.numpy()
        assert same_bits(ok.view(np.float32), ref)


# ----------------------------------------------------- the method steps -----

def test_delegates_match_brute_force():
    rng = _rng(6)
    for n, alpha, beta in [(1, 0, 1), (5, 1, 2), (37, 2, 2), (64, 3, 3), (100, 4, 4),
                           (257, 5, 2), (1000, 6, 1), (19, 3, 8)]:
        x = rng.integers(0, 6, n).astype(np.uint32)
        dk, di = oracle.delegates(x, alpha, beta)
        L = 1 << alpha
        S = (n + L - 1) // L
        assert dk.shape == (S, beta)
        for i in range(S):
            pos = sorted(range(i * L, min(n, (i + 1) * L)), key=lambda t: (-int(x[t]), t))
            for j in range(beta):
                if j < len(pos):
                    assert dk[i, j] == x[pos[j]] and di[i, j] == pos[j]
                else:
                    assert dk[i, j] == 0 and di[i, j] == -1


def test_threshold_is_kth_of_delegates():
    rng = _rng(7)
    x = rng.integers(0, 1000, 500).astype(np.uint32)
    dk, di = oracle.delegates(x, 3, 2)
    real = sorted(dk.ravel()[di.ravel() >= 0].tolist(), reverse=True)
    for k in (1, 2, 50, len(real)):
        assert oracle.threshold(dk, di, k) == real[k - 1]
    assert oracle.threshold(dk, di, len(real) + 1) == 0  # too few delegates


@pytest.mark.parametrize("kind", ["few", "rand", "asc", "desc", "equal"])
def test_candidates_and_method_equal_definition(kind):
    """Rules 1-3 keep exactly {x >= tau}, and the method's answer equals the
    plain definition, for every alpha and beta (Sec. 3)."""
    for seed in range(6):
        rng = _rng(200 + seed)
        n = int(rng.integers(1, 300))
        x = small_input(rng, n, kind, np.uint32)
        order = brute_order(x)
        for alpha in range(0, 7):
            for beta in (1, 2, 3, 4):
                dk, di = oracle.delegates(x, alpha, beta)
                for k in sorted({1, 2, n // 4 or 1, n // 2 or 1, n}):
                    tau = oracle.threshold(dk, di, k)
                    ck, ci, scanned = oracle.candidates(x, alpha, beta, dk, di, tau)
                    kth = int(x[order[k - 1]])
                    assert tau <= kth                                  # Rule 2
                    assert sorted(ci.tolist()) == [i for i in range(n) if x[i] >= tau]
                    assert np.array_equal(ck, x[ci])
                    assert len(ci) >= k
                    nd = int((dk[di >= 0] >= tau).sum())
                    assert scanned <= nd // beta                       # Rule 3
                    ok, oi, st = oracle.drtopk(x, oracle.U32, k, alpha, beta)
                    assert oi.tolist() == order[:k]
                    assert st["tau"] == tau and st["candidates"] == len(ci)


def test_method_equals_definition_typed():
    rng = _rng(9)
    for dtype in (np.int32, np.float32):
        for n in (50, 333):
            x = small_input(rng, n, "few", dtype)
            bits, dt = oracle.as_bits(x)
            for alpha, beta in [(2, 2), (4, 1), (5, 3)]:
                for k in (1, 7, n):
                    ref = oracle.topk(bits, dt, k)
                    got = oracle.drtopk(bits, dt, k, alpha, beta)
                    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_paper_worked_example():
    g = json.load(open(GOLDEN))
    v = np.array(g["V"], np.uint32)
    assert v.min() == g["min"] and v.max() == g["max"]
    assert int((v >= g["top_bucket_lo"]).sum()) == g["top_bucket_count"]
    a = g["alpha"]
    dk, di = oracle.delegates(v, a, 1)
    assert dk[:, 0].tolist() == g["D_beta1"]
    for c in g["cases"]:
        dk, di = oracle.delegates(v, a, c["beta"])
        tau = oracle.threshold(dk, di, c["k"])
        assert tau == c["tau"]
        ck, ci, scanned = oracle.candidates(v, a, c["beta"], dk, di, tau)
        assert sorted(ck.tolist()) == sorted(c["candidates"])
        assert scanned == len(c["scanned_subranges"])
        # which subranges were scanned: those whose beta delegates all reach tau
        sc = [i for i in range(dk.shape[0]) if dk[i, c["beta"] - 1] >= tau]
        assert sc == c["scanned_subranges"]
        if "qualified_subranges" in c:
            assert [i for i in range(dk.shape[0]) if dk[i, 0] >= tau] == c["qualified_subranges"]
        ok, oi, _ = oracle.drtopk(v, oracle.U32, c["k"], a, c["beta"])
        assert ok.tolist() == c["topk"]


# ------------------------------------------------------------- Rule 4 -------

def test_alpha_rule4_paper_value():
    # Sec. 4.3: |V| = 2^30, k = 2^24 gives alpha = 4 (from 4.5, rounded down)
    assert oracle.alpha_rule4(1 << 30, 1 << 24) == 4


def test_alpha_rule4_against_symbolic_eq6():
    sp = pytest.importorskip("sympy")
    a, V, k, Cg, Cs = sp.symbols("alpha V k C_g C_s", positive=True)
    # Eq. 6: T = 31 |V| 2^-a Cs + (6 |V| 2^-a + 6 k 2^a + 2k + |V|) Cg
    T = 31 * V * 2 ** (-a) * Cs + (6 * V * 2 ** (-a) + 6 * k * 2 ** a + 2 * k + V) * Cg
    sol = sp.solve(sp.Eq(sp.diff(T, a), 0), a)
    assert len(sol) == 1
    # Eq. 9 form: 1/2 [log2 V - log2 k + log2(6 Cg + 31 Cs) - log2(6 Cg)]
    eq9 = sp.Rational(1, 2) * (sp.log(V, 2) - sp.log(k, 2) + sp.log(6 * Cg + 31 * Cs, 2)
                               - sp.log(6 * Cg, 2))
    vals = {V: 2 ** 30, k: 2 ** 10, Cg: 3, Cs: 1}
    assert abs(float(sol[0].subs(vals)) - float(eq9.subs(vals))) < 1e-9
    assert float(sp.diff(T, a, 2).subs(vals).subs(a, 7)) > 0          # Eq. 7: convex
    # the oracle's rule is the Eq. 9 form with const = 3, rounded down
    c = 3.0
    for ln in range(1, 34, 3):
        for lk in range(0, ln + 1, 2):
            expr = 0.5 * (ln - lk + c)
            assert oracle.alpha_rule4(1 << ln, 1 << lk) == math.floor(expr)
    # non-powers of two
    assert oracle.alpha_rule4(3_000_000, 777) == math.floor(
        0.5 * (math.log2(3_000_000) - math.log2(777) + 3))


# ------------------------------------------------------- input recipes ------

def test_generator_hash_matches_reference_definition():
    for seed, stream in [(1, 0), (3, 6), (123456789, 21)]:
        h = inputs.hash_range(seed, stream, 1000, 64)
        ref = [inputs.hash_int(seed, stream, i) for i in range(1000, 1064)]
        got = [(int(v) + (1 << 64)) % (1 << 64) for v in h.tolist()]
        assert got == ref


def test_generator_recipes():
    n = 1 << 14
    asc = inputs.ascending_u32(n, 3).numpy().view(np.uint32)
    assert (np.diff(asc.astype(np.int64)) > 0).all()
    desc = inputs.descending_u32(n, 3).numpy().view(np.uint32)
    assert (np.diff(desc.astype(np.int64)) < 0).all()
    eq = inputs.all_equal_u32(n).numpy().view(np.uint32)
    assert (eq == inputs.ALL_EQUAL_VALUE).all()
    d16 = inputs.distinct16_u32(n, 3).numpy().view(np.uint32)
    assert len(np.unique(d16)) == 16
    assert sorted(np.unique(d16).tolist()) == sorted(inputs.distinct16_table(3))
    z = inputs.zipf_u32(1 << 16, 3).numpy().view(np.uint32).astype(np.int64)
    # mass at small values: P(v = 0) = 1 / zeta-like normaliser; small values dominate
    assert (z == 0).mean() > 0.05 and (z < 1000).mean() > 0.3 and z.max() > 1 << 20
    u = inputs.uniform_u32(1 << 16, 1).numpy().view(np.uint32).astype(np.float64)
    assert abs(u.mean() / 2 ** 32 - 0.5) < 0.01
    g = inputs.normal_f32(1 << 16, 2).numpy()
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1) < 0.02 and np.isfinite(g).all()
    pm = inputs.uniform_pm1_f32(1 << 16, 5).numpy()
    assert pm.min() >= -1 and pm.max() < 1
    # chunking does not change the stream
    a = inputs.uniform_u32(3000, 9)
    old = inputs.CHUNK
    try:
        inputs.CHUNK = 1000
        b = inputs.uniform_u32(3000, 9)
    finally:
        inputs.CHUNK = old
    assert torch.equal(a, b)


def test_batched_recipe():
    lens, ks = inputs.batched_rows(4096, 4)
    assert min(lens) >= 1 << 10 and max(lens) <= 1 << 22
    assert all(1 <= k <= min(1024, n) for n, k in zip(lens, ks))
    mean = sum(lens) / len(lens)
    # E[2^U[10,22]] = (2^22 - 2^10) / (12 ln 2) ~ 5.04e5
    assert 4.0e5 < mean < 6.2e5


# ------------------------------------------- smallest criterion, merge, omp ---

def brute_order_smallest(x):
    """Positions sorted by (value asc, index asc); -0.0 ranks below +0.0."""
    vals = x.tolist()
    if x.dtype == np.float32:
        def key(i):
            v = vals[i]
            poszero = 1 if (v == 0.0 and math.copysign(1.0, v) > 0) else 0
            return (v, poszero, i)
    else:
        def key(i):
            return (int(vals[i]), 0, i)
    return sorted(range(len(vals)), key=key)


@pytest.mark.parametrize("dtype", [np.uint32, np.int32, np.float32])
def test_bottomk_matches_brute_force_every_k(dtype):
    rng = _rng(61)
    for n in (1, 2, 3, 9, 40):
        for kind in ("few", "equal", "asc", "desc", "rand"):
            x = small_input(rng, n, kind, dtype)
            bits, dt = oracle.as_bits(x)
            order = brute_order_smallest(x)
            for k in range(1, n + 1):
                ok, oi = oracle.bottomk(bits, dt, k)
                assert oi.tolist() == order[:k], (n, kind, k)
                assert same_bits(ok, bits[order[:k]])
                assert oracle.kth_smallest(bits, dt, k) == int(bits[order[k - 1]])


def test_bottomk_special_cases():
    n = 50
    asc = np.arange(n, dtype=np.uint32) * 3
    ok, oi = oracle.bottomk(asc, oracle.U32, 7)
    assert oi.tolist() == list(range(7))
    ok, oi = oracle.bottomk(asc[::-1].copy(), oracle.U32, 7)
    assert oi.tolist() == list(range(n - 1, n - 8, -1))
    ok, oi = oracle.bottomk(np.full(n, 5, np.uint32), oracle.U32, 9)
    assert oi.tolist() == list(range(9))
    # k = 1 is the minimum at its first index
    x = np.array([4, 1, 9, 1, 0, 0, 3], np.uint32)
    ok, oi = oracle.bottomk(x, oracle.U32, 1)
    assert ok.tolist() == [0] and oi.tolist() == [4]


def test_bottomk_values_against_torch_on_distinct_keys():
    x = np.random.default_rng(62).permutation(5000).astype(np.int32) - 2500
    bits, dt = oracle.as_bits(x)
    for k in (1, 10, 999):
        ok, _ = oracle.bottomk(bits, dt, k)
        ref = torch.topk(torch.from_numpy(x.astype(np.int64)), k, largest=False).values
        assert oracle.from_bits(ok, dt).astype(np.int64).tolist() == sorted(ref.tolist())


def test_topk_merge_matches_brute_force():
    rng = _rng(63)
    for smallest in (False, True):
        for m in (1, 5, 60):
            keys = rng.integers(0, 4, m).astype(np.uint32)
            gidx = rng.permutation(10 * m)[:m].astype(np.int64)
            sign = 1 if smallest else -1
            order = sorted(range(m), key=lambda i: (sign * int(keys[i]), int(gidx[i])))
            for k in range(1, m + 1):
                ok, og = oracle.topk_merge(keys, gidx, oracle.U32, k, smallest)
                assert og.tolist() == [int(gidx[i]) for i in order[:k]], (m, k, smallest)
                assert ok.tolist() == [int(keys[i]) for i in order[:k]]


@pytest.mark.parametrize("smallest", [False, True])
def test_shard_topk_union_holds_the_answer(smallest):
    """The distributed form (Sec. 4.4): the top-k of the union of every
    shard's top-k equals the top-k of the whole vector, ties included."""
    rng = _rng(64)
    pick = oracle.bottomk if smallest else oracle.topk
    for kind in ("few", "rand"):
        n = 3001
        bits = (rng.integers(0, 6, n) if kind == "few"
                else rng.integers(0, 2**32, n, dtype=np.uint64)).astype(np.uint32)
        cuts = [0, 1, 700, 701, 1500, 3001]
        for k in (1, 5, 400, 1000):
            ck, cg = [], []
            for a, b in zip(cuts[:-1], cuts[1:]):
                kk = min(k, b - a)
                lk, li = pick(bits[a:b], oracle.U32, kk)
                ck.append(lk)
                cg.append(li.astype(np.int64) + a)
            ok, og = oracle.topk_merge(np.concatenate(ck), np.concatenate(cg), oracle.U32, k,
                                       smallest)
            rk, ri = pick(bits, oracle.U32, k)
            assert np.array_equal(ok, rk) and np.array_equal(og, ri.astype(np.int64)), (kind, k)


def test_topk_omp_equals_single_thread():
    rng = _rng(65)
    for n, kind in ((1, "rand"), (7, "few"), (1000, "few"), (100003, "rand"), (50000, "equal")):
        if kind == "few":
            bits = rng.integers(0, 3, n).astype(np.uint32)
        elif kind == "equal":
            bits = np.full(n, 9, np.uint32)
        else:
            bits = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
        for threads in (1, 3, 8):
            for k in sorted({1, min(n, 5), max(1, n // 3), n}):
                rk, ri = oracle.topk(bits, oracle.U32, k)
                ok, oi, used = oracle.topk_omp(bits, oracle.U32, k, threads)
                assert used == threads
                assert np.array_equal(ok, rk) and np.array_equal(oi, ri), (n, kind, threads, k)
