"""Parity at the full workload sizes, in the launch configuration the
benchmark times (default alpha/beta, one query per call).

* n = 2^28 float32 N(0, 1), k in {1, 32, 1024, 65536}: top-k and k-th
  compared with the CPU oracle element by element;
* n = 2^30 uint32, the five adversarial distributions, k in {1024, 2^20}:
  every query checked by properties that fix the exact answer (checked with
  plain torch reductions, independent of the library's kernels), and two
  queries also compared with the CPU oracle element by element.

The properties: the returned indices are distinct and hold the returned
keys; the output is sorted by (key desc, index asc); exactly the keys above
the k-th key are returned; the returned keys equal to the k-th key are the
smallest indices holding it. Together they leave one possible answer.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild
from paper_2109_08219_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def ordered_i64(t, dt):
    """Keys as int64 with the order of the key type (u32 bits held in int32)."""
    x = t.view(torch.int32).to(torch.int64)
    if dt == "u32":
        return x & 0xFFFFFFFF
    if dt == "i32":
        return x
    # f32: the order-preserving bit map, as a reduction-friendly int64
    u = x & 0xFFFFFFFF
    neg = (u >> 31) == 1
    return torch.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000)


def check_properties(x, dt, k, ok, oi):
    n = x.numel()
    idx = oi.to(torch.int64)
    assert idx.min().item() >= 0 and idx.max().item() < n
    assert torch.unique(idx).numel() == k
    assert torch.equal(x.view(torch.int32)[idx], ok.view(torch.int32))
    m = ordered_i64(ok, dt)
    # sorted by (key desc, index asc)
    dk = m[1:] - m[:-1]
    assert (dk <= 0).all()
    same = dk == 0
    assert (idx[1:][same] > idx[:-1][same]).all()
    kth = m[-1].item()
    mx = ordered_i64(x, dt)
    greater = int((mx > kth).sum().item())
    assert int((m > kth).sum().item()) == greater < k
    ties_needed = k - greater
    tie_pos = torch.nonzero(mx == kth).flatten()[:ties_needed]
    assert torch.equal(torch.sort(idx[m == kth]).values, tie_pos)


def test_f32_normal_2p28_against_oracle():
    dev = torch.device("cuda")
    n = 1 << 28
    x = inputs.normal_f32(n, 2, device=dev)
    bits = x.cpu().numpy().view(np.uint32)
    for k in (1, 32, 1024, 65536):
        ok, oi = drtopk.drtopk_topk(x, k)
        kth = drtopk.drtopk_kth(x, k)
        torch.cuda.synchronize()
        rk, ri = oracle.topk(bits, oracle.F32, k)
        assert np.array_equal(ok.cpu().numpy().view(np.uint32), rk), k
        assert np.array_equal(oi.cpu().numpy(), ri), k
        assert int(kth.cpu().numpy().view(np.uint32)[0]) == int(rk[-1])
        check_properties(x, "f32", k, ok, oi)


@pytest.mark.parametrize("dist", inputs.ADVERSARIAL)
def test_u32_adversarial_2p30_properties(dist):
    dev = torch.device("cuda")
    n = 1 << 30
    x = inputs.DISTRIBUTIONS[dist](n, 3, device=dev)
    for k in (1024, 1 << 20):
        ok, oi = drtopk.drtopk_topk(x, k, dtype="u32")
        kth = drtopk.drtopk_kth(x, k, dtype="u32")
        torch.cuda.synchronize()
        check_properties(x, "u32", k, ok, oi)
        assert int(kth.view(torch.int32).item()) == int(ok.view(torch.int32)[-1].item())
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dist,k", [("zipf", 1024), ("distinct16", 1 << 20)])
def test_u32_adversarial_2p30_against_oracle(dist, k):
    dev = torch.device("cuda")
    n = 1 << 30
    x = inputs.DISTRIBUTIONS[dist](n, 3, device=dev)
    ok, oi = drtopk.drtopk_topk(x, k, dtype="u32")
    torch.cuda.synchronize()
    bits = x.cpu().numpy().view(np.uint32)
    del x
    torch.cuda.empty_cache()
    rk, ri = oracle.topk(bits, oracle.U32, k)
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), rk)
    assert np.array_equal(oi.cpu().numpy(), ri)
