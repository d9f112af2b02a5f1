"""Device-side errors reach the caller, without any GPU fault.

Every wait inside a kernel is bounded; a wait that gives up records a flag,
and the last kernel of a query copies the flags to a per-device report word.
drtopk_wait_selftest launches one kernel whose bounded wait runs out (it
waits on an mbarrier phase nothing completes, with the wait the bulk-copy
rings use) and reports it the same way. The tests check that the timeout
comes back as DRTOPK_ERR_TIMEOUT through drtopk_sync_status, through the
next asynchronous query call and through the synchronous host entry point,
exactly once, and that the context stays usable.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild

pytestmark = pytest.mark.gpu

TIMEOUT = 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def host_bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def data(n=100003, seed=3):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    return b, torch.from_numpy(b.view(np.int32)).cuda()


def test_sync_status_reports_a_timed_out_wait_once():
    drtopk.sync_status()  # start clean
    drtopk.wait_selftest(2000)
    with pytest.raises(drtopk.DrTopkError) as e:
        drtopk.sync_status()
    assert e.value.status == TIMEOUT
    drtopk.sync_status()  # cleared
    b, x = data()
    ok, oi = drtopk.drtopk_topk(x, 100, dtype="u32")
    drtopk.sync_status()
    rk, ri = oracle.topk(b, oracle.U32, 100)
    assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)


def test_next_query_reports_it_then_queries_run():
    drtopk.sync_status()
    b, x = data(seed=4)
    ok = torch.empty(50, dtype=torch.int32, device="cuda")
    oi = torch.empty(50, dtype=torch.int32, device="cuda")
    for _ in range(3):  # plain launches, then graph replays of the same query
        drtopk.drtopk_topk(x, 50, out_keys=ok, out_idx=oi, dtype="u32")
    drtopk.wait_selftest(1000)
    torch.cuda.synchronize()
    with pytest.raises(drtopk.DrTopkError) as e:
        drtopk.drtopk_topk(x, 50, out_keys=ok, out_idx=oi, dtype="u32")
    assert e.value.status == TIMEOUT
    # reported once: the following calls run and report nothing
    kt = drtopk.drtopk_kth(x, 50, dtype="u32")
    drtopk.drtopk_topk(x, 50, out_keys=ok, out_idx=oi, dtype="u32")
    drtopk.sync_status()
    rk, ri = oracle.topk(b, oracle.U32, 50)
    assert np.array_equal(host_bits(ok), rk) and np.array_equal(oi.cpu().numpy(), ri)
    assert int(host_bits(kt)[0]) == int(rk[-1])


def test_host_entry_point_reports_it():
    drtopk.sync_status()
    b, _ = data(seed=5)
    drtopk.wait_selftest(1000)
    torch.cuda.synchronize()
    with pytest.raises(drtopk.DrTopkError) as e:
        drtopk.drtopk_topk_host(b, 10, "u32")
    assert e.value.status == TIMEOUT
    ok, oi = drtopk.drtopk_topk_host(b, 10, "u32")
    rk, ri = oracle.topk(b, oracle.U32, 10)
    assert np.array_equal(ok, rk) and np.array_equal(oi, ri)


def test_selftest_argument_checks():
    with pytest.raises(drtopk.DrTopkError):
        drtopk.wait_selftest(0)
    with pytest.raises(drtopk.DrTopkError):
        drtopk.wait_selftest(10**8)
