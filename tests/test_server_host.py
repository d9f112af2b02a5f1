"""Host-only logic of the server: the bytes a request counts against the
HBM budget, the batched-or-single routing, and argument checks made before
any CUDA call. No GPU needed."""

import ctypes

import pytest

import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return drtopk.lib()


def test_footprint_and_routing(L):
    # small rows are batched: keys + outputs only (the batch scratch is the
    # server's own)
    b, batched = drtopk.server_footprint(1 << 16, 100)
    assert batched and b == 4 * (1 << 16) + 8 * 100
    # above batch_max_n (default 2^20) or k > 4096: a single query with its workspace
    _, _, ws = drtopk.drtopk_plan(1 << 22, 100)
    b, batched = drtopk.server_footprint(1 << 22, 100)
    assert not batched and b == 4 * (1 << 22) + 8 * 100 + ws
    b, batched = drtopk.server_footprint(1 << 16, 5000)
    assert not batched
    # a larger batch_max_n batches more; the plain flag batches nothing
    assert drtopk.server_footprint(1 << 22, 100, batch_max_n=1 << 22)[1]
    assert not drtopk.server_footprint(1 << 12, 10, flags=drtopk.SERVER_PLAIN)[1]


def test_footprint_argument_checks(L):
    fp = lambda *a: L.drtopk_server_footprint(*a, None, None)
    assert fp(0, 0, 1, 0, 0) == 1          # n = 0
    assert fp(0, 10, 11, 0, 0) == 2        # k > n
    assert fp(0, 10, 0, 0, 0) == 2         # k = 0
    assert fp(9, 10, 1, 0, 0) == 3         # dtype
    assert fp(0, 1 << 31, 1, 0, 0) == 1    # n > 2^31 - 1


def test_server_calls_reject_null_handles(L):
    t = ctypes.c_uint64()
    assert L.drtopk_server_submit(None, None, 0, 1, 1, None, None, ctypes.byref(t)) == 1
    assert L.drtopk_server_poll_ex(None, 1, None) == 1
    assert L.drtopk_server_destroy(None) == 1
    h = ctypes.c_void_p()
    assert L.drtopk_server_create_ex(1 << 30, -1, 0, 0, ctypes.byref(h)) == 1
    assert L.drtopk_server_create_ex(1 << 30, 0, 4, 0, ctypes.byref(h)) == 1  # unknown flag
