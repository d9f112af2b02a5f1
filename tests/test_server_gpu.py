"""The served form: every request's result is bit-identical to the same
request run alone (drtopk_topk), whatever it was mixed with; admission keeps
the admitted device-resident state within the HBM budget; requests larger
than the budget are refused; submissions from several host threads and a
destroy with requests still queued all complete correctly. Some requests are
also checked against the CPU oracle."""

import threading

import numpy as np
import pytest
import torch

import oracle
import paper_2109_08219_gb300 as drtopk
from paper_2109_08219_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DT = {"u32": oracle.U32, "i32": oracle.I32, "f32": oracle.F32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    drtopk.lib()


def make_requests(count, seed, lo=10, hi=22, kmax_exp=14):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(round(2.0 ** rng.uniform(lo, hi)))
        k = min(n, int(round(2.0 ** rng.uniform(0, kmax_exp))))
        dt = ["u32", "i32", "f32"][i % 3]
        if rng.random() < 0.5:
            x = torch.randn(n, device="cuda")
            if dt != "f32":
                x = (x * 1e6).to(torch.int32)
        else:
            x = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device="cuda")
            if dt == "f32":
                x = torch.rand(n, device="cuda")
        if i % 7 == 0:   # heavy ties
            x = x // 1000 if x.dtype == torch.int32 else torch.round(x * 4) / 4
        ok = torch.empty(k, dtype=x.dtype, device="cuda")
        oi = torch.empty(k, dtype=torch.int32, device="cuda")
        reqs.append((x, k, dt, ok, oi))
    return reqs


def alone(x, k, dt):
    return drtopk.drtopk_topk(x, k, dtype=dt)


def check_same(reqs, refs):
    for i, ((x, k, dt, ok, oi), (rk, ri)) in enumerate(zip(reqs, refs)):
        assert torch.equal(ok.view(torch.int32), rk.view(torch.int32)), i
        assert torch.equal(oi, ri), i


@pytest.mark.parametrize("plain", [False, True])
def test_mixed_equals_alone(plain):
    reqs = make_requests(160, 1 if not plain else 2)
    refs = [alone(x, k, dt) for x, k, dt, _, _ in reqs]
    torch.cuda.synchronize()
    with drtopk.Server(16 << 30, plain=plain) as srv:
        tickets = [srv.submit(x, k, ok, oi, dtype=dt) for x, k, dt, ok, oi in reqs]
        lats = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert all(l > 0 for l in lats)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    if plain:
        assert st["batches"] == 0 and st["single_queries"] == len(reqs)
    else:
        assert st["batches"] >= 1 and st["batched_requests"] >= 1
        assert st["batched_requests"] + st["single_queries"] == len(reqs)
    check_same(reqs, refs)
    # a few against the CPU oracle
    for x, k, dt, ok, oi in reqs[:12]:
        bits = x.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)
        rk, ri = oracle.topk(bits, DT[dt], k)
        assert np.array_equal(ok.cpu().view(torch.int32).numpy().view(np.uint32), rk)
        assert np.array_equal(oi.cpu().numpy(), ri)


def test_budget_bounds_admitted_state():
    reqs = make_requests(60, 3, lo=18, hi=24, kmax_exp=12)
    refs = [alone(x, k, dt) for x, k, dt, _, _ in reqs]
    torch.cuda.synchronize()
    fps = [drtopk.server_footprint(x.numel(), k, dt)[0] for x, k, dt, _, _ in reqs]
    probe = drtopk.Server(8 << 30)
    fixed = probe.stats()["fixed_bytes"]
    probe.close()
    budget = fixed + 2 * max(fps)   # about two requests at a time
    with drtopk.Server(budget) as srv:
        tickets = [srv.submit(x, k, ok, oi, dtype=dt) for x, k, dt, ok, oi in reqs]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
        assert st["peak_bytes"] <= budget
        assert st["completed"] == len(reqs)
        # a request larger than the budget is refused at submission
        big = torch.empty(1 << 27, device="cuda")
        okb = torch.empty(10, device="cuda")
        oib = torch.empty(10, dtype=torch.int32, device="cuda")
        if drtopk.server_footprint(big.numel(), 10)[0] > budget - fixed:
            with pytest.raises(drtopk.DrTopkError) as e:
                srv.submit(big, 10, okb, oib)
            assert e.value.status == 6
    check_same(reqs, refs)


def test_threads_and_destroy_with_queued_requests():
    reqs = make_requests(120, 4, lo=10, hi=20)
    refs = [alone(x, k, dt) for x, k, dt, _, _ in reqs]
    torch.cuda.synchronize()
    srv = drtopk.Server(16 << 30)
    errors = []

    def worker(part):
        try:
            for x, k, dt, ok, oi in part:
                srv.submit(x, k, ok, oi, dtype=dt)
        except Exception as ex:  # surfaced below
            errors.append(ex)

    ths = [threading.Thread(target=worker, args=(reqs[i::4],)) for i in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errors
    srv.close()   # drains every queued request
    torch.cuda.synchronize()
    check_same(reqs, refs)


def test_poll_states():
    x = torch.randn(1 << 20, device="cuda")
    ok = torch.empty(64, device="cuda")
    oi = torch.empty(64, dtype=torch.int32, device="cuda")
    with drtopk.Server(8 << 30) as srv:
        t = srv.submit(x, 64, ok, oi)
        lat = None
        while lat is None:
            lat = srv.poll(t)
        assert lat > 0
        with pytest.raises(drtopk.DrTopkError):   # forgotten after completion
            srv.poll(t)
    rk, ri = drtopk.drtopk_topk(x, 64)
    assert torch.equal(ok, rk) and torch.equal(oi, ri)
