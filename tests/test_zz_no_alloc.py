"""drtopk_kth_noalloc: k-selection for callers that may not allocate device
memory at query time (allocation forbidden after start-up, or device memory
wholly owned by another allocator). It runs on the library's fixed 64 MiB
device array; its answers must equal drtopk_kth's, call after call, even
though every call reuses (and finds stale) the same scratch.

Kept in its own file, collected last."""

import numpy as np
import pytest
import torch

import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def bits(t):
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def test_noalloc_matches_kth_on_consecutive_calls():
    dev = torch.device("cuda")
    cases = [
        (inputs.uniform_u32(1 << 20, 1, device=dev), "u32", 128),
        (inputs.distinct16_u32(3 << 18, 2, device=dev), "u32", 4000),
        (inputs.normal_f32(1 << 22, 3, device=dev), "f32", 1024),
        (inputs.all_equal_u32(100003, device=dev), "u32", 77),
        (inputs.zipf_u32(1 << 21, 4, device=dev), "u32", 1),
    ]
    for x, dt, k in cases:
        ref = drtopk.drtopk_kth(x, k, dtype=dt)
        a = drtopk.drtopk_kth_noalloc(x, k, dtype=dt)
        b = drtopk.drtopk_kth_noalloc(x, k, dtype=dt)  # second call in a row
        torch.cuda.synchronize()
        assert bits(a)[0] == bits(ref)[0], (dt, k)
        assert bits(b)[0] == bits(ref)[0], (dt, k)


def test_noalloc_full_size_and_limit():
    dev = torch.device("cuda")
    x = inputs.uniform_u32(1 << 28, 7, device=dev)
    for k in (1, 1024, 4096):
        ref = drtopk.drtopk_kth(x, k, dtype="u32")
        got = drtopk.drtopk_kth_noalloc(x, k, dtype="u32")
        torch.cuda.synchronize()
        assert bits(got)[0] == bits(ref)[0]
    with pytest.raises(drtopk.DrTopkError) as e:
        drtopk.drtopk_kth_noalloc(x, 1 << 20, dtype="u32")  # needs far more than 64 MiB
    assert e.value.status == 4
