"""Host-only logic of the batched form: argument checks of a batch plan and
the per-shape tuning table. No compute call: these run without a GPU."""

import ctypes

import numpy as np
import pytest

import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return drtopk.lib()


def create(L, off, ks, alpha=0, beta=0, dtype=0):
    off = np.ascontiguousarray(off, np.int64)
    ks = np.ascontiguousarray(ks, np.int32)
    h = ctypes.c_void_p()
    rc = L.drtopk_batch_plan_create(dtype, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    int(ks.size), alpha, beta, ctypes.byref(h))
    if rc == 0:
        L.drtopk_batch_plan_destroy(h)
    return rc


def test_plan_argument_checks(L):
    assert create(L, [0, 10], [0]) == 2                  # k = 0
    assert create(L, [0, 10], [11]) == 2                 # k > n
    assert create(L, [0, 10000], [4097]) == 2            # k above the batched limit
    assert create(L, [0, 10, 10], [1, 1]) == 1           # empty row
    assert create(L, [0, 10, 5], [1, 1]) == 1            # decreasing offsets
    assert create(L, [-4, 10], [1]) == 1                 # negative start
    assert create(L, [0, (1 << 24) + 1], [1]) == 1       # row above 2^24 keys
    assert create(L, [0, 10], [1], dtype=5) == 3         # dtype
    assert create(L, [0, 10], [1], alpha=4) == 1         # alpha below 5
    assert create(L, [0, 10], [1], alpha=17) == 1
    assert create(L, [0, 10], [1], beta=5) == 1
    h = ctypes.c_void_p()
    assert L.drtopk_batch_plan_create(0, None, None, 1, 0, 0, ctypes.byref(h)) == 1
    assert L.drtopk_batch_plan_run(None, None, None, None, None) == 1
    assert L.drtopk_batch_plan_destroy(None) == 1


def test_tuning_table_roundtrip(L):
    assert drtopk.tune_get(20, 10) == (0, 0)
    drtopk.tune_set(20, 10, 1, 0)              # direct select
    assert drtopk.tune_get(20, 10) == (1, 0)   # untouched: Rule 4
    drtopk.tune_set(20, 10, 9, 3)
    assert drtopk.tune_get(20, 10) == (9, 3)
    drtopk.tune_set(20, 10, 0, 0)
    assert drtopk.tune_get(20, 10) == (0, 0)
    for bad in [(9, 0, 5, 1), (32, 0, 5, 1), (20, 13, 5, 1), (20, 3, 4, 1), (20, 3, 17, 1),
                (20, 3, 5, 5), (20, 3, 5, -1)]:
        with pytest.raises(drtopk.DrTopkError):
            drtopk.tune_set(*bad)
    with pytest.raises(drtopk.DrTopkError):
        drtopk.tune_get(40, 0)


def test_batch_limits(L):
    lim = drtopk.batch_limits()
    assert lim["max_k"] == 4096 and lim["max_row"] == 1 << 24 and lim["direct_max"] == 4096
    assert lim["max_delegates"] >= 4096 and lim["onchip_candidates"] >= 2048
    assert lim["direct_max_onchip"] >= lim["direct_max"]
