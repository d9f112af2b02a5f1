"""The exactness argument of the speculative compaction of the delegate
vector, checked on the CPU with the oracle's own delegates (Rules 1 and 3)
and threshold (Rule 2), independently of the CUDA path.

For a bound t, the records are the subranges whose largest delegate m^0 is
>= t, each with all of its beta delegates. The claims the GPU path relies on:
  1. every delegate >= t belongs to a record;
  2. if at least k delegates are >= t, then tau (the k-th largest delegate)
     is >= t, and the k-th largest key among the recorded delegates is tau;
  3. every subrange with m^0 > tau is recorded (so classifying only the
     records finds every subrange Rules 1-3 keep);
  4. if fewer than k delegates are >= t, then tau < t (the fallback case).
Bounds are taken around tau, at quantiles of the delegates and at the
extremes, on inputs with distinct keys, few distinct values, sorted and
clustered keys, for beta in 1..4 and several alpha and k.
"""

import numpy as np
import pytest

import oracle


def inputs(n, seed):
    rng = np.random.default_rng(seed)
    yield "uniform", rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    yield "few", rng.integers(0, 6, n).astype(np.uint32) * np.uint32(0x01000193)
    yield "ascending", np.arange(n, dtype=np.uint32) * np.uint32(3)
    yield "descending", (np.arange(n, dtype=np.uint32) * np.uint32(3))[::-1].copy()
    clustered = rng.integers(0, 1 << 12, n).astype(np.uint32)
    for c in range(0, n, 4096):
        clustered[c:c + 64] = rng.integers(1 << 31, 1 << 32, min(64, n - c), dtype=np.uint64)
    yield "clustered", clustered


def kth_largest(v, k):
    return int(np.sort(v)[::-1][k - 1])


@pytest.mark.parametrize("beta", [1, 2, 3, 4])
def test_records_hold_tau_and_every_kept_subrange(beta):
    n = 50000
    checked = 0
    for name, bits in inputs(n, 40 + beta):
        mapped = oracle.map_keys(bits, oracle.U32)
        for alpha in (5, 6, 8):
            dk, di = oracle.delegates(mapped, alpha, beta)
            dk = dk.astype(np.int64)
            real = di >= 0                         # padded slots of short subranges
            flat = dk[real]
            for k in (1, 7, 100, min(flat.size, 2000)):
                if k > flat.size:
                    continue
                tau = oracle.threshold(dk, di, k)
                assert tau == kth_largest(flat, k)
                q = np.quantile(flat, [0.0, 0.5, 0.9, 0.99]).astype(np.uint64)
                bounds = {0, int(tau), max(0, int(tau) - 1), int(tau) + 1,
                          int(flat.max()), *(int(x) for x in q)}
                for t in bounds:
                    rec = dk[:, 0] >= t                # records: m^0 >= t
                    vals = dk[rec][real[rec]]          # their delegates
                    above = int(np.sum(flat >= t))
                    # 1: every delegate >= t is recorded
                    assert int(np.sum(vals >= t)) == above, (name, alpha, k, t)
                    if above >= k:
                        # 2: tau >= t and the k-th largest recorded key is tau
                        assert tau >= t
                        assert kth_largest(vals, k) == tau, (name, alpha, k, t)
                        # 3: every subrange with m^0 > tau is recorded
                        assert np.all(rec[dk[:, 0] > tau])
                    else:
                        # 4: tau below the bound (the fallback writes the full arrays)
                        assert tau < t
                    checked += 1
    assert checked > 100


def test_sampled_bound_is_conservative_on_uniform_input():
    """The sample's rule (1.5x the expected count above tau, plus 8 standard
    deviations and 64) picks a bound below tau on uniform keys: the sampled
    chunks' delegates, scaled by the sampled share, estimate the count of
    delegates above any bound."""
    rng = np.random.default_rng(7)
    n, alpha, beta, chunk, stride = 1 << 22, 6, 2, 8192, 128
    bits = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    dk, di = oracle.delegates(bits, alpha, beta)
    sub_per_chunk = chunk >> alpha
    sampled = np.zeros(dk.shape[0], bool)
    for c in range(0, n // chunk, stride):
        sampled[c * sub_per_chunk:(c + 1) * sub_per_chunk] = True
    samp = dk[sampled].ravel()
    for k in (1 << 10, 1 << 14, 1 << 16):
        target = k * samp.size / dk.size
        need = 1.5 * target + 8.0 * np.sqrt(target) + 64.0
        bins = np.bincount((samp >> 21).astype(np.int64), minlength=2048)
        cum = np.cumsum(bins[::-1])                # from the top bin down
        top = int(np.argmax(cum >= need))          # bins from the top
        t = (2047 - top) << 21
        tau = oracle.threshold(dk, di, k)
        assert int(np.sum(dk.ravel() >= t)) >= k and tau >= t, k


def test_plan_reserves_records_only_for_eligible_shapes():
    """drtopk_plan's workspace includes the records of the speculative
    compaction (S/4 records of beta keys, beta segments and a subrange id)
    exactly for arrays of 2^26 keys or more with alpha in [5, 10]."""
    import paper_2109_08219_gb300 as drtopk
    from paper_2109_08219_gb300 import build as libbuild
    libbuild.build()

    def al(b):
        return (b + 255) // 256 * 256

    for n, k in (((1 << 26), 1 << 16), ((1 << 30), 1 << 20), ((1 << 28), 1 << 14)):
        a, b, ws = drtopk.drtopk_plan(n, k)
        assert 5 <= a <= 10
        a2, b2, ws_small = drtopk.drtopk_plan(n - 1, k)   # one key short of eligible at 2^26
        S = (n + (1 << a) - 1) >> a
        rec = max(1024, S // 4)
        extra = al(rec * b * 4) + al(rec * b * 2) + al(rec * 4)
        if n == 1 << 26:
            assert (a2, b2) == (a, b) and ws - ws_small >= extra - 4096
    # alpha above 10 (small k): no records
    a, b, ws = drtopk.drtopk_plan(1 << 30, 1024)
    assert a == 11
    a3, b3, ws3 = drtopk.drtopk_plan((1 << 30) - 1, 1024)
    assert abs(ws - ws3) < 1 << 20
