#!/usr/bin/env python3
"""Benchmark of delegate-centric top-k on GB300 (one JSON line on stdout).

Workload (default): exact top-k over n = 2^30 uint32 keys, five adversarial
distributions for delegate filtering (ascending, descending, all-equal, 16
distinct values, Zipf(1.1) over [0, 2^32)) and k in {1024, 2^20}. One step
= the 10 queries, inputs resident in HBM (4 GiB each, larger than L2, so no
flush is needed). value = keys processed / second (Gkeys/s) over all ranks.

Extra measurements in the same line:
  roofline      delegate pass (the kernel that streams all n keys):
                algorithmic bytes 4n per launch / mean CUDA-event duration on
                the launching stream, against MEASURED_PEAKS.json hbm_gbs;
  e2e           same metric through drtopk_topk_host (host keys in pinned
                memory, H2D copy and D2H of the results inside the timing);
  cpu_baseline  the CPU oracle (single thread) on a bounded sample;
  clocks        nvidia-smi samples taken during the timed region;
  breakdown     per (distribution, k): ms, candidates kept, stage times;
  batched       the ragged batch (4096 float32 rows, lengths round(2^U[10,22]),
                k_r uniform in [1, min(1024, n_r)], N(0,1)) in one graph-replayed
                persistent launch, default and autotuned parameters, against the
                same rows as 4096 plain per-row calls (and those calls captured in
                one CUDA graph);
  ablations     candidate-ratio curves on UD (n in 2^24..2^30, k in 2^4..2^20)
                and, at n = 2^30 on UD and ND, the method against beta = 1
                (Rules 1+2 alone), Rule 2's filtering off, and the first select
                stopped one digit early (all exact);
  served        Poisson arrivals of float32 requests (n log-uniform in
                [2^12, 2^28], k log-uniform in [1, 2^14], N(0,1) or U[-1,1)
                by coin flip) at offered loads {0.25 .. 1.2} x the plain mode's
                measured saturation rate through the server
                (64 GB HBM budget) and through its plain mode (one launch
                sequence per request, one stream): throughput, p50 / p99 latency.

--impl reference times the CPU oracle instead (the chunked multi-core
variant on all host cores, rank 0 only).
Multi-GPU (torchrun): the distributed form of Sec. 4.4. Rank r holds the r-th
2^log2n-key sub-vector of each query's vector; per query every rank computes
its local top-k, the lists are all-gathered (NCCL) and rank 0 computes the
exact final top-k with drtopk_topk_merge. Weak scaling: value = keys of all
ranks over the slowest rank's time.
"""

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DISTS = ["ascending", "descending", "all_equal", "distinct16", "zipf"]
KS = [1024, 1 << 20]
SEED = 3
PAPER_UD_MS = 6.4  # Dr. Top-k radix, |V| = 2^30 UD, k = 1024, V100S (Sec. 5.1)
# DRAM bytes (read + write) per key of one delegate-pass launch, by alpha
# (the subrange size sets the delegate writes): ncu dram__bytes_read.sum +
# dram__bytes_write.sum of the delegate kernel in this benchmark's own
# launches at n = 2^30 (Zipf input, k = 1024 -> alpha 11, k = 2^20 ->
# alpha 6; mean of two launches each). Must be re-measured (or set to None)
# whenever the delegate kernel changes.
# DRAM bytes (read + write) of a query's delegate stage per key at n = 2^30,
# by (alpha, delegate path), from one ncu capture of this benchmark's
# launches (dram__bytes_read.sum + dram__bytes_write.sum, one pass):
#   path 0: the full delegate pass alone;
#   path 1: sample (1/128 of the chunks) + records pass + idle fallback;
#   path 2: sample + idle records pass + the fallback as the full pass;
#   path 3: records, then the full pass again (the sample misled: rare).
DELEG_DRAM_BYTES_PER_KEY = {(11, 0): 4301.0e6 / (1 << 30),
                            (6, 0): 4446.1e6 / (1 << 30),
                            (6, 1): 4335.8e6 / (1 << 30),
                            (6, 2): 4480.8e6 / (1 << 30),
                            (6, 3): (4335.8e6 + 4446.1e6) / (1 << 30)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="drtopk", choices=["drtopk", "reference"])
    ap.add_argument("--log2n", type=int, default=30)
    ap.add_argument("--dists", default=",".join(DISTS))
    ap.add_argument("--ks", default=",".join(str(k) for k in KS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip breakdown/context runs")
    ap.add_argument("--no-batched", action="store_true", help="skip the ragged batch")
    ap.add_argument("--no-served", action="store_true", help="skip the served workload")
    ap.add_argument("--no-ablations", action="store_true",
                    help="skip the candidate-ratio curves and the ablations")
    ap.add_argument("--batched-rows", type=int, default=4096,
                    help="rows of the ragged batch (the first rows of the 4096-row recipe)")
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="arrivals per offered load")
    return ap.parse_args()


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.samples = []
        self.proc = None
        self.index = index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [s for (t, s) in self.samples if t0 - 0.15 <= t <= t1 + 0.15]
        if not rows and self.samples:
            # the timed region is shorter than the sampling period: nearest sample
            mid = 0.5 * (t0 + t1)
            rows = [min(self.samples, key=lambda ts: abs(ts[0] - mid))[1]]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------- distributed ----
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_seed(rank):
    """Seed of rank r's sub-vector (rank 0: the one-GPU workload's seed)."""
    return SEED + 1000 * rank


def aggregate_value(n, queries, steps, world, ms_max):
    """Whole-job Gkeys/s: keys of all ranks over the slowest rank's time."""
    return float(n) * queries * steps * world / (ms_max * 1e-3) / 1e9


# ------------------------------------------------------------ oracle leg ---
def oracle_sample(dists, ks, sample_log2, reps=1, data=None):
    """Single-thread CPU oracle over the first 2^sample_log2 keys of each query
    (the generators are element-wise in the index, so a prefix of the full
    input is the same array at the smaller size)."""
    import numpy as np
    import oracle
    from paper_2109_08219_gb300 import inputs
    m = 1 << sample_log2
    if data is None:
        data = {d: inputs.DISTRIBUTIONS[d](m, SEED).numpy().view(np.uint32) for d in dists}
    oracle.topk(data[dists[0]][:1024], oracle.U32, 1)  # load the library
    keys = 0
    t = 0.0
    for _ in range(reps):
        for d in dists:
            for k in ks:
                kk = min(k, m)
                t0 = time.perf_counter()
                oracle.topk(data[d], oracle.U32, kk)
                t += time.perf_counter() - t0
                keys += m
    return keys, t


def oracle_sample_omp(dists, ks, data, reps=1):
    """The chunked multi-core oracle (all host cores) on the same samples."""
    import oracle
    keys, t, used = 0, 0.0, 1
    first = next(iter(data.values()))
    oracle.topk_omp(first[:4096], oracle.U32, 1)  # start the thread pool
    for _ in range(reps):
        for d in dists:
            for k in ks:
                x = data[d]
                t0 = time.perf_counter()
                _, _, used = oracle.topk_omp(x, oracle.U32, min(k, x.size))
                t += time.perf_counter() - t0
                keys += x.size
    return keys, t, used


def cpu_model():
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def e2e_sharded(drtopk, shard, x_dev, ks, n, world, rank, dev, args):
    """End to end on several ranks through the public API: every step copies
    each rank's sub-vector from pinned host memory to its GPU, runs the
    sharded top-k (local drtopk_select, all-gather, drtopk_topk_merge on
    rank 0) and reads the merged result back to the host on rank 0. One
    distribution (the first), every k; max over ranks."""
    import torch
    host = torch.empty(n, dtype=torch.int32, pin_memory=True)
    host.copy_(x_dev)
    dbuf = torch.empty(n, dtype=torch.int32, device=dev)
    outs_h = {k: (torch.empty(k, dtype=torch.int32, pin_memory=True),
                  torch.empty(k, dtype=torch.int64, pin_memory=True)) for k in ks}

    def estep():
        for k in ks:
            dbuf.copy_(host, non_blocking=True)
            r = shard.shard_topk(dbuf, k, dtype="u32")
            if r is not None:
                outs_h[k][0].copy_(r[0], non_blocking=True)
                outs_h[k][1].copy_(r[1], non_blocking=True)
        torch.cuda.synchronize()

    estep()
    esteps = max(2, min(args.steps, 5))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(esteps):
        estep()
    et = max_over_ranks(time.perf_counter() - t0, world)
    del dbuf, host
    torch.cuda.empty_cache()
    return {"value": float(n) * world * len(ks) * esteps / et / 1e9, "unit": "Gkeys/s",
            "h2d_bytes_per_step": 4 * n * world * len(ks),
            "d2h_bytes_per_step": 12 * sum(ks), "steps": esteps,
            "api": "per rank: pinned H2D copy of the sub-vector, drtopk_select, all-gather, "
                   "drtopk_topk_merge on rank 0, D2H of the merged keys and int64 indices",
            "workload": "first distribution only, every k"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    dists = args.dists.split(",")
    ks = [int(x) for x in args.ks.split(",")]
    import numpy as np
    from paper_2109_08219_gb300 import inputs
    sample_log2 = min(21, args.log2n)
    m = 1 << sample_log2
    data = {d: inputs.DISTRIBUTIONS[d](m, SEED).numpy().view(np.uint32) for d in dists}
    for _ in range(args.warmup):
        oracle_sample_omp(dists, ks, data)
    keys, t, used = oracle_sample_omp(dists, ks, data, reps=args.steps)
    gk = keys / t / 1e9
    sample = ("first 2^%d keys of each of the %d (distribution, k) queries, %d steps; chunked "
              "oracle (per-thread nth_element, then the union), %d threads"
              % (sample_log2, len(dists) * len(ks), args.steps, used))
    out = {
        "impl": "reference",
        "metric": "top-k throughput (n=2^%d u32, adversarial distributions)" % args.log2n,
        "value": gk, "unit": "Gkeys/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": workload_config(args, dists, ks, world),
        "cpu_baseline": {"value": gk, "unit": "Gkeys/s", "cores": used, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": gk, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def workload_config(args, dists, ks, world=1):
    cfg = {"workload": "top-k, n=2^%d uint32 keys, distributions %s, k in %s, 1 query per "
                       "(distribution, k) per step" % (args.log2n, "/".join(dists),
                                                      "/".join(str(k) for k in ks)),
           "n": 1 << args.log2n, "k": ks, "distributions": dists, "seed": SEED,
           "queries_per_step": len(dists) * len(ks),
           "l2": "inputs larger than L2 (%d MiB each); no flush" % ((4 << args.log2n) >> 20),
           "parallelism": "single GPU"}
    if world > 1:
        cfg["parallelism"] = ("shard + gather over %d GPUs (Sec. 4.4): rank r holds the r-th "
                              "sub-vector (2^%d keys, seed %d + 1000 r) of a %d x 2^%d-key "
                              "vector; per query a local top-k, one all-gather of the k-entry "
                              "lists and the exact merge on rank 0"
                              % (world, args.log2n, SEED, world, args.log2n))
    return cfg


# ----------------------------------------------------------------- main ----
# -------------------------------------------------------------- batched ----
def batched_measure(drtopk, inputs, dev, peak, rows=4096, reps=10):
    import numpy as np
    import torch
    lens, ks = inputs.batched_rows(rows, 4)
    row_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(row_off[-1])
    ksn = np.array(ks, np.int32)
    x = inputs.normal_f32(total, 4, device=dev)
    out = {"workload": "%d float32 rows, len round(2^U[10,22]), k_r U{1..min(1024,n_r)}, "
                       "N(0,1), seed 4" % rows, "keys": total, "rows": rows,
           "inputs_larger_than_L2": True}

    def time_plan(tag):
        plan = drtopk.BatchPlan(row_off, ksn, "f32")
        ok = torch.empty(plan.total_k, dtype=torch.float32, device=dev)
        oi = torch.empty(plan.total_k, dtype=torch.int32, device=dev)
        s = torch.cuda.Stream(dev)
        with torch.cuda.stream(s):
            for _ in range(3):
                plan.run(x, ok, oi, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.run(x, ok, oi, stream=s)
        plan.phase_cycles(reset=True, stream=s)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            for _ in range(reps):
                g.replay()
            e1.record(s)
        s.synchronize()
        plan.status(s)
        ms = e0.elapsed_time(e1) / reps
        cyc = plan.phase_cycles(stream=s)
        a, b = plan.params()
        plan.close()
        tot = float(sum(cyc.values())) or 1.0
        out[tag] = {"ms": ms, "gkeys_s": total / ms / 1e6, "gbs": 4.0 * total / ms / 1e6,
                    "hbm_frac_of_measured": 4.0 * total / ms / 1e6 / peak,
                    "kernels_per_batch": 1,
                    "direct_rows": int((a == 0).sum()),
                    "cycle_share": {k: round(v / tot, 4) for k, v in cyc.items()}}
        return ok, oi

    ok0, oi0 = time_plan("rule4")
    t0 = time.perf_counter()
    # two rows per SM: at least one per CTA of the batched launch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    drtopk.autotune_batched("f32", 12, 22, rows_per_shape=2 * sms)
    out["autotune_s"] = time.perf_counter() - t0
    ok1, oi1 = time_plan("autotuned")
    out["autotuned_equals_rule4"] = bool(torch.equal(ok0.view(torch.int32), ok1.view(torch.int32))
                                         and torch.equal(oi0, oi1))
    # the same rows as one plain call each
    oo = np.concatenate([[0], np.cumsum(ksn.astype(np.int64))])
    pk = torch.empty(int(oo[-1]), dtype=torch.float32, device=dev)
    pi = torch.empty(int(oo[-1]), dtype=torch.int32, device=dev)

    def per_row():
        for r in range(rows):
            a, b, o, k = int(row_off[r]), int(row_off[r + 1]), int(oo[r]), int(ksn[r])
            drtopk.drtopk_topk(x[a:b], k, out_keys=pk[o:o + k], out_idx=pi[o:o + k])

    per_row()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    per_row()
    e1.record()
    torch.cuda.synchronize()
    out["per_row_plain_ms"] = e0.elapsed_time(e1)
    out["per_row_equals_batched"] = bool(torch.equal(pk.view(torch.int32), ok0.view(torch.int32))
                                         and torch.equal(pi, oi0))
    try:
        s = torch.cuda.Stream(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            per_row()
        with torch.cuda.stream(s):
            g.replay()
            e0.record(s)
            g.replay()
            g.replay()
            e1.record(s)
        s.synchronize()
        out["per_row_graph_ms"] = e0.elapsed_time(e1) / 2
        del g
    except Exception as ex:  # report, do not fail the bench
        out["per_row_graph_ms"] = None
        out["per_row_graph_error"] = repr(ex)[:200]
    best = min(out["rule4"]["ms"], out["autotuned"]["ms"])
    out["speedup_vs_per_row_plain"] = out["per_row_plain_ms"] / best
    if out.get("per_row_graph_ms"):
        out["speedup_vs_per_row_graph"] = out["per_row_graph_ms"] / best
    del x, pk, pi
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ ablations ----
def ablations_measure(drtopk, inputs, dev, reps=3):
    import torch
    out = {"curves_workload": "UD u32 (seed 1), prefixes of one 2^30 array", "curves": [],
           "ablations_workload": "n = 2^30 u32, UD (seed 1) and ND = round(N(1e8, 10)) (seed 1)",
           "ablations": []}
    ud = inputs.uniform_u32(1 << 30, 1, device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    for ln in (24, 26, 28, 30):
        n = 1 << ln
        x = ud[:n]
        for lk in (4, 10, 16, 20):
            k = 1 << lk
            ok = torch.empty(k, dtype=torch.int32, device=dev)
            oi = torch.empty(k, dtype=torch.int32, device=dev)
            ms, _ = timed(lambda: drtopk.drtopk_topk(x, k, out_keys=ok, out_idx=oi, dtype="u32"))
            _, _, _, st = drtopk.drtopk_topk_ex(x, k, want_kth=False, dtype="u32")
            cand = st["greater"] + st["ties_needed"]
            out["curves"].append({
                "log2n": ln, "log2k": lk, "ms": ms, "gkeys_s": n / ms / 1e6,
                "alpha": st["alpha"], "beta": st["beta"], "candidate_fraction": cand / n,
                "workload_fraction": (st["beta"] * st["subranges"] + cand) / n,
                "scanned_subranges": st["scanned"]})
    nd = inputs.nd_u32(1 << 30, 1, device=dev)
    variants = [("method", {}), ("beta1_rules_1_2", {"beta": 1}),
                ("rule2_filter_off", {"no_filter": True}),
                ("first_select_skips_last_digit", {"skip_last_digit": True})]
    s = torch.cuda.Stream(dev)
    for name, x in (("UD", ud), ("ND", nd)):
        for k in (1024, 1 << 20):
            ok = torch.empty(k, dtype=torch.int32, device=dev)
            oi = torch.empty(k, dtype=torch.int32, device=dev)
            for vname, kw in variants:
                # every variant the same way: its launches captured in one CUDA
                # graph and replayed; statistics read by a separate call
                def call():
                    drtopk.drtopk_topk_ablate(x, k, dtype="u32", stats=False, out_keys=ok,
                                              out_idx=oi, stream=s, **kw)
                with torch.cuda.stream(s):
                    call()
                s.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    call()
                with torch.cuda.stream(s):
                    g.replay()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    for _ in range(reps):
                        g.replay()
                    e1.record(s)
                s.synchronize()
                ms = e0.elapsed_time(e1) / reps
                del g
                st = drtopk.drtopk_topk_ablate(x, k, dtype="u32", **kw)[2]
                cand = st["greater"] + st["ties_needed"]
                out["ablations"].append({
                    "input": name, "k": k, "variant": vname, "ms": ms,
                    "alpha": st["alpha"], "beta": st["beta"], "tau": st["tau"],
                    "candidate_fraction": cand / x.numel(),
                    "scanned_subranges": st["scanned"]})
    out["ablations_timing"] = ("each variant's call captured in one CUDA graph and replayed "
                               "(mean of %d replays); statistics read outside the timed loop" % reps)
    del ud, nd
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------- served ----
def served_measure(drtopk, dev, arrivals, budget=64 << 30, pool=192, seed=5):
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    for _ in range(pool):
        n = int(round(2.0 ** rng.uniform(12, 28)))
        k = min(n, int(round(2.0 ** rng.uniform(0, 14))))
        if rng.random() < 0.5:
            x = torch.randn(n, device=dev, generator=g)
        else:
            x = torch.rand(n, device=dev, generator=g) * 2 - 1
        reqs.append((x, k))
    kmax = max(k for _, k in reqs)
    mean_keys = float(np.mean([x.numel() for x, _ in reqs]))
    order = rng.integers(0, pool, arrivals)
    outs = [(torch.empty(kmax, device=dev), torch.empty(kmax, dtype=torch.int32, device=dev))
            for _ in range(arrivals)]
    torch.cuda.synchronize()

    def run(plain, rate):
        """rate None: all requests at once (closed loop, capacity)."""
        srv = drtopk.Server(budget, device=dev.index or 0, plain=plain)
        # warm-up: one of each request shape class
        for i in range(min(8, pool)):
            x, k = reqs[i]
            srv.wait(srv.submit(x, k, outs[i][0], outs[i][1]))
        gaps = rng.exponential(1.0 / rate, arrivals) if rate else np.zeros(arrivals)
        t_arr = np.cumsum(gaps)
        tickets = []
        t0 = time.perf_counter()
        for j in range(arrivals):
            while time.perf_counter() - t0 < t_arr[j]:
                pass
            x, k = reqs[order[j]]
            tickets.append(srv.submit(x, k, outs[j][0], outs[j][1]))
        lats = [srv.wait(t) for t in tickets]
        t1 = time.perf_counter()
        st = srv.stats()
        srv.close()
        lats = np.sort(np.array(lats))
        keys = float(sum(reqs[i][0].numel() for i in order))
        return {"offered_rps": rate, "achieved_rps": arrivals / (t1 - t0),
                "gkeys_s": keys / (t1 - t0) / 1e9,
                "p50_us": float(lats[len(lats) // 2]),
                "p99_us": float(lats[min(len(lats) - 1, int(0.99 * len(lats)))]),
                "mean_us": float(lats.mean()), "batches": st["batches"],
                "batched_requests": st["batched_requests"],
                "peak_gb": st["peak_bytes"] / 1e9}

    cap_server = run(False, None)
    cap_plain = run(True, None)
    loads = []
    base = cap_plain["achieved_rps"]
    for frac in (0.25, 0.5, 0.75, 0.9, 1.0, 1.2):
        rate = frac * base
        loads.append({"offered_frac_of_plain_capacity": frac,
                      "server": run(False, rate), "plain": run(True, rate)})
    del reqs, outs
    torch.cuda.empty_cache()
    return {"workload": "Poisson arrivals, float32, n log-uniform [2^12, 2^28], k log-uniform "
                        "[1, 2^14], N(0,1) or U[-1,1) by coin flip, %d distinct requests "
                        "(mean n %.3g), %d arrivals per load" % (pool, mean_keys, arrivals),
            "budget_gb": budget / 2**30, "latency": "submit to completion seen by the scheduler",
            "capacity": {"server": cap_server, "plain": cap_plain}, "loads": loads}


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch
    import paper_2109_08219_gb300 as drtopk
    from paper_2109_08219_gb300 import build as libbuild
    from paper_2109_08219_gb300 import inputs
    from paper_2109_08219_gb300 import shard

    libbuild.build()
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)
    dists = args.dists.split(",")
    ks = [int(x) for x in args.ks.split(",")]
    n = 1 << args.log2n
    # one GPU: the whole vector of each query; several (torchrun): rank r
    # holds the r-th contiguous sub-vector of a vector of world * n keys
    xs = {d: inputs.DISTRIBUTIONS[d](n, shard_seed(rank), device=dev) for d in dists}
    outs = {k: (torch.empty(k, dtype=torch.int32, device=dev),
                torch.empty(k, dtype=torch.int32, device=dev)) for k in ks}
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def step():
        for d in dists:
            for k in ks:
                if world == 1:
                    drtopk.drtopk_topk(xs[d], k, out_keys=outs[k][0], out_idx=outs[k][1],
                                       dtype="u32", stream=stream)
                else:
                    # Sec. 4.4: local top-k, all-gather of the lists, merge on rank 0
                    shard.shard_topk(xs[d], k, dtype="u32", stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clk = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    if clk is not None:
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = drtopk.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    launches = drtopk.launch_count() - launches0
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world)
    if clk is not None:
        time.sleep(0.2)
        clk.stop()
    # Stage profile: the same workload again with per-stage CUDA events on
    # the launching stream (profiled calls launch kernel by kernel instead of
    # replaying the cached graph of the query; the kernels are the same).
    psteps = max(1, min(args.steps, 20))
    drtopk.profile_begin()
    ep0 = torch.cuda.Event(enable_timing=True)
    ep1 = torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    for _ in range(psteps):
        step()
    ep1.record(stream)
    torch.cuda.synchronize()
    prof = drtopk.profile_end()
    prof_ms_step = ep0.elapsed_time(ep1) / psteps
    queries = len(dists) * len(ks)
    value = aggregate_value(n, queries, args.steps, world, ms_max)

    e2e_dist = None
    if world > 1 and not args.no_e2e:
        e2e_dist = e2e_sharded(drtopk, shard, xs[dists[0]], ks, n, world, rank, dev, args)
    if rank != 0:
        return

    # roofline of the delegate pass
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    if not peak:
        peak = 6800.0
    dms, dl = prof["delegate"]
    achieved = (4.0 * n) / ((dms / max(dl, 1)) * 1e-3) / 1e9 if dl else None
    # DRAM traffic of the timed delegate stages: each query's alpha and
    # delegate path (from its statistics, read outside the timed region)
    # pick the measured bytes per key; the mean over the timed queries
    paths = {}
    for d in dists:
        for k in ks:
            st = drtopk.drtopk_topk_ex(xs[d], k, want_kth=False, dtype="u32")[3]
            paths[(d, k)] = (st["alpha"], st["delegate_path"])
    per_q = {"%s/k=%d" % dk: {"alpha": ap[0], "path": ap[1],
                              "bytes": (DELEG_DRAM_BYTES_PER_KEY.get(ap) or 0) * n or None}
             for dk, ap in paths.items()}
    traffic = (sum(q["bytes"] for q in per_q.values()) / len(per_q)
               if all(q["bytes"] for q in per_q.values()) else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_by_query": per_q,
                "traffic_ratio_to_4n_by_alpha_path": {
                    "%d/%d" % ap: v * n / (4.0 * n) for ap, v in DELEG_DRAM_BYTES_PER_KEY.items()},
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                  "delegate stage's kernels per (alpha, delegate path), "
                                  "captured in this benchmark's launches at n=2^30; mean over "
                                  "the timed queries",
                "kernel": "delegate stage: delegate_kernel (TMA-streamed delegate pass; for "
                          "alpha <= 10 on large arrays a sampled bound and a records pass)",
                "algorithmic_bytes_per_launch": 4 * n, "launches": dl,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs, copy burst)" % peak_src,
                "frac_vs_nominal_8TBps": (achieved / 8000.0) if achieved else None,
                "end_to_end_frac_of_peak": (4.0 * n * queries * args.steps / (ms * 1e-3) / 1e9) / peak}
    stage_ms = {k: (v[0] / max(v[1], 1)) for k, v in prof.items()}

    out = {
        "metric": "top-k throughput (n=2^%d u32, adversarial distributions)" % args.log2n,
        "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args, dists, ks, world),
        "roofline": roofline,
        "gpu_launches": launches,
        "stage_ms_per_query": stage_ms,
        "stage_profile": {"steps": psteps, "ms_per_step": prof_ms_step,
                          "note": "second timed region, same workload, kernel-by-kernel launches "
                                  "with per-stage CUDA events; roofline.achieved comes from it"},
    }
    if clk is not None:
        out["clocks"] = clk.summary(tw0, tw1)

    # breakdown per query + candidate statistics + context UD line
    if not args.no_extra:
        bd = []
        for d in dists:
            for k in ks:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                reps = 5
                e0.record(stream)
                for _ in range(reps):
                    drtopk.drtopk_topk(xs[d], k, out_keys=outs[k][0], out_idx=outs[k][1],
                                       dtype="u32", stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                qms = e0.elapsed_time(e1) / reps
                _, _, _, st = drtopk.drtopk_topk_ex(xs[d], k, want_kth=False, dtype="u32")
                bd.append({"dist": d, "k": k, "ms": qms, "gkeys_s": n / qms / 1e6,
                           "alpha": st["alpha"], "beta": st["beta"],
                           "candidate_fraction": (st["greater"] + st["ties_needed"]) / n,
                           "workload_fraction": (st["beta"] * st["subranges"] + st["greater"]
                                                 + st["ties_needed"]) / n,
                           "greater": st["greater"], "ties_needed": st["ties_needed"],
                           "scanned_subranges": st["scanned"],
                           "tie_scanned_subranges": st["tie_scanned"]})
        out["breakdown"] = bd
        # context: the paper's headline setting (UD, k = 1024) on this GPU
        ud = inputs.uniform_u32(n, 1, device=dev)
        o1 = (torch.empty(1024, dtype=torch.int32, device=dev),
              torch.empty(1024, dtype=torch.int32, device=dev))
        for _ in range(3):
            drtopk.drtopk_topk(ud, 1024, out_keys=o1[0], out_idx=o1[1], dtype="u32")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            drtopk.drtopk_topk(ud, 1024, out_keys=o1[0], out_idx=o1[1], dtype="u32")
        e1.record(stream)
        torch.cuda.synchronize()
        ums = e0.elapsed_time(e1) / 20
        out["context_uniform_k1024"] = {
            "ms": ums, "gkeys_s": n / ums / 1e6, "hbm_frac_of_measured": (4.0 * n / ums / 1e6) / peak,
            "paper_ms_v100s": PAPER_UD_MS if args.log2n == 30 else None,
            "note": "paper number is V100S (1134 GB/s), context only"}
        del ud

    if not args.no_ablations and world == 1:
        out["ablations"] = ablations_measure(drtopk, inputs, dev)
    if not args.no_batched and world == 1:
        out["batched"] = batched_measure(drtopk, inputs, dev, peak, rows=args.batched_rows)
    if not args.no_served and world == 1:
        out["served"] = served_measure(drtopk, dev, args.served_requests)

    if not args.no_cpu and world == 1:
        sample_log2 = min(26, args.log2n)
        m = 1 << sample_log2
        data = {d: xs[d][:m].cpu().numpy().view(np.uint32) for d in dists}
        keys, t = oracle_sample(dists, ks, sample_log2, data=data)
        mkeys, mt, used = oracle_sample_omp(dists, ks, data)
        out["cpu_baseline"] = {
            "value": mkeys / mt / 1e9, "unit": "Gkeys/s", "cores": used, "kind": "oracle",
            "sample": "first 2^%d keys of each of the %d (distribution, k) queries, once "
                      "(chunked oracle: per-thread nth_element, then nth_element + sort of "
                      "the union, %d threads)" % (sample_log2, queries, used),
            "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
            "single_thread": {"value": keys / t / 1e9, "unit": "Gkeys/s", "cores": 1,
                              "sample": "same keys, std::nth_element + sort, 1 thread"}}

    if e2e_dist is not None:
        out["e2e"] = e2e_dist
    # end to end through the host entry point
    if not args.no_e2e and world == 1:
        hosts = {}
        for d in dists:
            h = torch.empty(n, dtype=torch.int32, pin_memory=True)
            h.copy_(xs[d])
            hosts[d] = h
        hk = {k: (torch.empty(k, dtype=torch.int32, pin_memory=True),
                  torch.empty(k, dtype=torch.int32, pin_memory=True)) for k in ks}
        # free the device copies: the host path stages its own
        del xs
        torch.cuda.empty_cache()

        # the host link alone: one H2D copy of each pinned input (the bound
        # of any path that must move the keys to the GPU)
        stage = torch.empty(n, dtype=torch.int32, device=dev)
        stage.copy_(hosts[dists[0]], non_blocking=True)
        torch.cuda.synchronize()
        link_gbs = 0.0
        for _ in range(2):  # best of two rounds
            t0 = time.perf_counter()
            for d in dists:
                stage.copy_(hosts[d], non_blocking=True)
            torch.cuda.synchronize()
            link_gbs = max(link_gbs, 4.0 * n * len(dists) / (time.perf_counter() - t0) / 1e9)
        del stage
        torch.cuda.empty_cache()

        call_s = []

        def estep():
            for d in dists:
                for k in ks:
                    c0 = time.perf_counter()
                    drtopk.drtopk_topk_host_ptr(hosts[d].data_ptr(), n, k, "u32",
                                                hk[k][0].data_ptr(), hk[k][1].data_ptr())
                    call_s.append(time.perf_counter() - c0)
        for _ in range(2):  # warm-up rounds (the first calls after set-up are slower)
            estep()
        esteps = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        call_s.clear()
        t0 = time.perf_counter()
        for _ in range(esteps):
            estep()
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        cms = sorted(1e3 * c for c in call_s)
        med = cms[len(cms) // 2]
        # the slow calls by (round, query in round): a pattern points at the
        # library, scattered ones at the shared host
        slow = [[j // queries, j % queries, round(1e3 * c, 2)] for j, c in enumerate(call_s)
                if 1e3 * c > 1.5 * med][:16]
        out["e2e"] = {"value": float(n) * queries * esteps / et / 1e9, "unit": "Gkeys/s",
                      "h2d_bytes_per_step": 4 * n * queries,
                      "d2h_bytes_per_step": 8 * sum(ks) * len(dists),
                      "steps": esteps, "api": "drtopk_topk_host (pinned host keys; copies in "
                      "~128 MB pieces overlapped with the delegate pass)",
                      "h2d_link_gbs": link_gbs,
                      "link_bound_gkeys": link_gbs / 4.0,
                      "frac_of_link_bound": (float(n) * queries * esteps / et / 1e9) / (link_gbs / 4.0),
                      "frac_of_link_bound_median_call": (4.0 * n / (med * 1e-3) / 1e9) / link_gbs,
                      "call_ms": {"min": cms[0], "median": med, "max": cms[-1],
                                  "calls": len(cms),
                                  "above_1.5x_median": sum(c > 1.5 * med for c in cms),
                                  "slow_calls_round_query_ms": slow}}

    print(json.dumps(out))


if __name__ == "__main__":
    main()
