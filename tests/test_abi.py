"""The C ABI library: builds, loads, exports every declared symbol, and its
host-only logic (argument checks, Rule 4 parameter choice) behaves. No
compute call is made here: these run without a GPU."""

import ctypes
import os
import re

import pytest

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "drtopk.h")


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return drtopk.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(drtopk_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("drtopk_kth", "drtopk_topk", "drtopk_plan", "drtopk_status_str",
                 "drtopk_topk_ex", "drtopk_delegates", "drtopk_topk_host"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    raw = ctypes.CDLL(drtopk.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), name


def test_status_strings(L):
    for i, name in enumerate(drtopk.STATUS):
        assert drtopk.status_str(i) == name
    assert drtopk.status_str(99) == "DRTOPK_UNKNOWN_STATUS"


def test_argument_checks_happen_before_cuda(L):
    p = ctypes.c_void_p(0x1000)  # never dereferenced: checks fail first
    out = ctypes.c_void_p(0x2000)
    assert L.drtopk_topk(p, 0, 100, 0, out, out, None) == 2          # k = 0
    assert L.drtopk_topk(p, 0, 100, 101, out, out, None) == 2        # k > n
    assert L.drtopk_topk(p, 0, 0, 1, out, out, None) == 1            # n = 0
    assert L.drtopk_topk(p, 0, 1 << 31, 1, out, out, None) == 1      # n > 2^31 - 1
    assert L.drtopk_topk(p, 7, 100, 1, out, out, None) == 3          # dtype
    assert L.drtopk_topk(None, 0, 100, 1, out, out, None) == 1       # null keys
    assert L.drtopk_topk(ctypes.c_void_p(0x1002), 0, 100, 1, out, out, None) == 1  # misaligned
    assert L.drtopk_topk(p, 0, 100, 1, None, out, None) == 1         # null output
    assert L.drtopk_kth(p, 0, 100, 1, None, None) == 1
    assert L.drtopk_topk_ex(p, 0, 100, 5, 1, 2, out, out, None, None, None) == 1  # alpha < 2
    assert L.drtopk_topk_ex(p, 0, 100, 5, 4, 5, out, out, None, None, None) == 1  # beta > 4
    assert L.drtopk_delegates(p, 0, 100, 1, 2, out, out, None) == 1
    assert L.drtopk_delegates(p, 0, 100, 2, 5, out, out, None) == 1


def test_plan_follows_rule4(L):
    # Rule 4 / Eq. 9 with const = 3 and floor, where the clamps do not bind
    for ln in range(12, 32):
        for lk in range(0, ln - 3):
            n, k = (1 << ln) - (1 if ln == 31 else 0), 1 << lk
            a, b, ws = drtopk.drtopk_plan(n, k)
            assert b == 2
            ref = oracle.alpha_rule4(n, k)
            S_ref = (n + (1 << ref) - 1) >> ref if 2 <= ref <= 16 else None
            if 2 <= ref <= 16 and 2 * S_ref >= 2 * k:
                assert a == ref, (ln, lk, a, ref)
            assert 2 <= a <= 16
            assert ws > 0


def test_plan_paper_value(L):
    # Sec. 4.3: |V| = 2^30, k = 2^24 -> alpha = 4
    assert drtopk.drtopk_plan(1 << 30, 1 << 24)[0] == 4
    assert drtopk.drtopk_plan(1 << 30, 1024)[0] == 11
    assert drtopk.drtopk_plan(1 << 30, 1 << 20)[0] == 6


def test_plan_keeps_enough_delegates(L):
    for n, k in [(100, 60), (5000, 2000), (1 << 20, 1 << 19), (7, 7)]:
        a, b, _ = drtopk.drtopk_plan(n, k)
        S = (n + (1 << a) - 1) >> a
        assert a == 2 or b * S >= 2 * k


def test_plan_rejects_bad_sizes(L):
    with pytest.raises(drtopk.DrTopkError):
        drtopk.drtopk_plan(10, 11)
    with pytest.raises(drtopk.DrTopkError):
        drtopk.drtopk_plan(0, 1)


def test_ablation_argument_checks(L):
    p = ctypes.c_void_p(0x1000)
    out = ctypes.c_void_p(0x2000)
    assert L.drtopk_topk_ablate(p, 0, 100, 1, 0, 0, 4, out, out, None, None) == 1   # flag
    assert L.drtopk_topk_ablate(p, 0, 100, 1, -1, 0, 1, out, out, None, None) == 1  # alpha
    assert L.drtopk_topk_ablate(p, 0, 100, 0, 0, 0, 1, out, out, None, None) == 2   # k = 0
    assert L.drtopk_topk_ablate(p, 0, 100, 1, 0, 0, 1, None, out, None, None) == 1  # outputs


def test_select_merge_and_selftest_check_arguments_before_cuda(L):
    """drtopk_select, drtopk_topk_merge and drtopk_wait_selftest reject bad
    arguments with a status before any CUDA call (no GPU here)."""
    p = ctypes.c_void_p(0x1000)  # never dereferenced
    out = ctypes.c_void_p(0x2000)
    # drtopk_select(keys, dtype, n, k, flags, out_keys, out_idx, out_kth, stream)
    assert L.drtopk_select(p, 0, 100, 5, 2, out, out, None, None) == 1     # unknown flag
    assert L.drtopk_select(p, 0, 100, 5, 0, out, None, None, None) == 1    # keys without idx
    assert L.drtopk_select(p, 0, 100, 5, 0, None, None, None, None) == 1   # no output
    assert L.drtopk_select(p, 9, 100, 5, 1, out, out, None, None) == 3     # dtype
    assert L.drtopk_select(p, 0, 100, 0, 1, out, out, None, None) == 2     # k = 0
    assert L.drtopk_select(p, 0, 100, 101, 1, None, None, out, None) == 2  # k > n

    def arr(v):
        a = (ctypes.c_int64 * len(v))(*v)
        return ctypes.cast(a, ctypes.POINTER(ctypes.c_int64)), a

    def merge(off, base, k, parts=None, flags=0, dtype=0, keys=p):
        po, _ka = arr(off)
        pb, _kb = arr(base)
        n = len(off) - 1 if parts is None else parts
        return L.drtopk_topk_merge(keys, p, dtype, po, pb, n, k, flags, out, out, None)

    assert merge([0, 5, 10], [0, 100], 3, keys=None) == 1       # null keys
    assert merge([0, 5, 10], [0, 100], 3, parts=0) == 1         # no parts
    assert merge([0] * 258, [0] * 257, 1, parts=257) == 1       # more than 256 parts
    assert merge([0, 5, 10], [0, 100], 3, flags=4) == 1         # unknown flag
    assert merge([0, 5, 10], [0, 100], 3, dtype=9) == 3         # dtype
    assert merge([0, 6, 5], [0, 100], 3) == 1                   # offsets decrease
    assert merge([0, 5, 10], [0, -1], 3) == 1                   # negative base
    assert merge([4, 4, 4], [0, 100], 1) == 1                   # empty lists
    assert merge([0, 5, 10], [0, 100], 11) == 2                 # k > listed entries
    assert merge([0, 5, 10], [0, 100], 0) == 2                  # k = 0
    # the selftest's wait limit: 1 us to 10 s
    assert L.drtopk_wait_selftest(0, None) == 1
    assert L.drtopk_wait_selftest(10000001, None) == 1
    assert drtopk.alloc_count() >= 0
