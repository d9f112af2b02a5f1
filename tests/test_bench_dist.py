"""The benchmark's multi-process path on CPU (gloo, world size 2): rank
barrier, max-over-ranks timing, the weak-scaling aggregate, and the
reference arm under torchrun (rank 0 prints the one JSON line, the other
rank exits 0 without work). Replicas only: no data-path collective."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    out.put((rank, m, bench.aggregate_value(1 << 20, 10, 3, w, m)))
    dist.destroy_process_group()


def test_gloo_two_ranks_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    # both ranks see the max of their times; value = keys of all ranks / max time
    assert [m for _, m, _ in res] == [15.0, 15.0]
    expect = (1 << 20) * 10 * 3 * 2 / (15.0e-3) / 1e9
    assert all(v == pytest.approx(expect) for _, _, v in res)


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % free_port(), "bench.py",
           "--impl", "reference", "--gpus", "2", "--log2n", "16", "--steps", "1",
           "--warmup", "1", "--dists", "zipf", "--ks", "64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
