"""drtopk_kth_noalloc: k-selection for callers that may not allocate device
memory at query time (allocation forbidden after start-up, or device memory
wholly owned by another allocator). It runs on the library's fixed 64 MiB
device array; its answers must equal the oracle's and drtopk_kth's, call
after call, even though every call reuses (and finds stale) the same
scratch; and a run of calls must allocate nothing.

Kept in its own file, collected last."""

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu

DT = {"u32": oracle.U32, "i32": oracle.I32, "f32": oracle.F32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def test_noalloc_matches_oracle_and_kth_on_consecutive_calls():
    dev = torch.device("cuda")
    cases = [
        (inputs.uniform_u32(1 << 20, 1, device=dev), "u32", 128),
        (inputs.distinct16_u32(3 << 18, 2, device=dev), "u32", 4000),
        (inputs.normal_f32(1 << 22, 3, device=dev), "f32", 1024),
        (inputs.all_equal_u32(100003, device=dev), "u32", 77),
        (inputs.zipf_u32(1 << 21, 4, device=dev), "u32", 1),
        (inputs.uniform_u32(777777, 5, device=dev), "i32", 999),
        (inputs.nd_u32(1 << 21, 6, device=dev), "i32", 4096),
    ]
    for x, dt, k in cases:
        want = oracle.kth(bits(x), DT[dt], k)
        ref = drtopk.drtopk_kth(x, k, dtype=dt)
        a = drtopk.drtopk_kth_noalloc(x, k, dtype=dt)
        b = drtopk.drtopk_kth_noalloc(x, k, dtype=dt)  # second call in a row
        torch.cuda.synchronize()
        assert bits(ref)[0] == want, (dt, k)
        assert bits(a)[0] == want, (dt, k)
        assert bits(b)[0] == want, (dt, k)
    drtopk.sync_status()  # no device-side error was reported


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the array's address and may load
    the module), a run of calls changes neither the library's allocation
    count nor the device's free memory nor torch's allocator state."""
    dev = torch.device("cuda")
    xs = [(inputs.uniform_u32(1 << 22, 8, device=dev), "u32", 4096),
          (inputs.normal_f32(1 << 21, 9, device=dev), "f32", 1),
          (inputs.distinct16_u32(1 << 20, 10, device=dev), "i32", 300)]
    outs = [torch.empty(1, dtype=x.dtype, device=dev) for x, _, _ in xs]
    for (x, dt, k), o in zip(xs, outs):
        drtopk.drtopk_kth_noalloc(x, k, out=o, dtype=dt)
    torch.cuda.synchronize()
    allocs0 = drtopk.alloc_count()
    free0, _ = torch.cuda.mem_get_info()
    torch0 = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    for _ in range(5):
        for (x, dt, k), o in zip(xs, outs):
            drtopk.drtopk_kth_noalloc(x, k, out=o, dtype=dt)
    torch.cuda.synchronize()
    assert drtopk.alloc_count() == allocs0
    assert torch.cuda.mem_get_info()[0] == free0
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == torch0
    for (x, dt, k), o in zip(xs, outs):
        assert bits(o)[0] == oracle.kth(bits(x), DT[dt], k), (dt, k)


def test_noalloc_full_size_and_limit():
    dev = torch.device("cuda")
    x = inputs.uniform_u32(1 << 28, 7, device=dev)
    hb = bits(x)
    # small and medium k first
    for k in (1, 1024, 4096):
        got = drtopk.drtopk_kth_noalloc(x, k, dtype="u32")
        torch.cuda.synchronize()
        assert bits(got)[0] == oracle.kth(hb, oracle.U32, k), k
    with pytest.raises(drtopk.DrTopkError) as e:
        drtopk.drtopk_kth_noalloc(x, 1 << 20, dtype="u32")  # needs far more than 64 MiB
    assert e.value.status == 4

    # a query at the edge of the array: bisect for a k that fits while k + 1
    # does not (a call that does not fit returns DRTOPK_ERR_NOMEM before any
    # launch), then check that k against the oracle
    def fits(k):
        try:
            drtopk.drtopk_kth_noalloc(x, k, dtype="u32")
            return True
        except drtopk.DrTopkError as err:
            assert err.status == 4
            return False
    lo, hi = 4096, 1 << 20
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    got = drtopk.drtopk_kth_noalloc(x, lo, dtype="u32")
    torch.cuda.synchronize()
    assert bits(got)[0] == oracle.kth(hb, oracle.U32, lo), lo
    drtopk.sync_status()
