"""Benchmark of the GB300 ε-distance self-join (one JSON line on rank 0).

Workload: the paper-scale synthetic configuration -- 2,000,000 points i.i.d.
uniform in [0,1)^d, FP64, ε per d chosen (by the CPU oracle, offline) for 32
mean neighbours, k chosen automatically.  A step runs the whole hot path on
each listed d: REORDER, grid index, adjacent-cell search, SHORTC distances (or
the tensor-core filter + FP64 recheck) and result emission into a device
buffer.  Metric: distance evaluations per second, where one evaluation is one
unordered candidate pair of the paper's grid at the chosen k (points in
adjacent cells, i < j; here the grid holds every pair), the unit fixed by the
index and independent of the kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form plain|tc]
                  [--dims 16,32,64] [--impl ours|reference]

--impl reference times the CPU oracle (test infrastructure, plain C) on a
bounded sample of the same workload.  Under torchrun each rank joins the
entity partition (Sec. 6.2) part=rank of N (no data-path collective; only the
timing max and the counts are reduced).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = os.path.join(ROOT, "tests", "golden", "workloads.json")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--form", choices=["plain", "tc"], default="tc")
    ap.add_argument("--workload", choices=["paper", "jobs", "exponential", "qe"], default="paper",
                    help="paper: 2M uniform points per d; jobs: the 256 uneven jobs in one launch; "
                         "exponential: the paper's own Syn16/32/64D2M shape (exponential, lambda = 40); "
                         "qe: the similarity join Q join_eps E, 200k queries against the 2M d=16 set")
    ap.add_argument("--nq", type=int, default=200_000, help="queries of the qe workload")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the one-shot plain FP64 join of the d=16 set beside the tc form")
    ap.add_argument("--plain-full", action="store_true",
                    help="run the plain FP64 join over the whole set at every listed d (minutes at d = 32 "
                         "and 64) instead of timing a 1/32 part of the d = 32 and 64 sets")
    ap.add_argument("--dims", default=None, help="comma list of d for the paper-scale workload")
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-budget", type=float, default=None,
                    help="reference arm: seconds of CPU work per step (default: sized so that the whole "
                         "run takes about 2.5 minutes, 3-20 s per step)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="build with the analytic k instead of the autotuner's picks")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------

def rank_max(dist, x: float, device: str = "cuda") -> float:
    """The maximum of x over the ranks (the step time: the slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_sum(dist, xs: list, device: str = "cuda") -> list:
    """Element-wise sums over the ranks (per-rank pair counts of the entity
    partition add up to |R|: the parts are disjoint)."""
    if dist is None:
        return list(xs)
    import torch
    t = torch.tensor([int(v) for v in xs], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]


def settings_of(t) -> dict:
    """Index settings from one autotuner pick (None: the analytic k)."""
    if not t:
        return {"k": 0}
    return {"k": t["k"], "query_block": t["query_block"], "tile": t["tile"]}


def agree(dist, obj):
    """Rank 0's value of obj on every rank.  The autotuner times trials, so
    two ranks tuning on their own may pick different k or query blocks; the
    entity partition deals parts of one load-ordered item list, so every rank
    must build with the same picks (Sec. 6.2)."""
    if dist is None:
        return obj
    box = [obj]
    dist.broadcast_object_list(box, src=0)
    return box[0]


def check_same(dist, obj, what: str) -> None:
    """Raise on every rank unless all ranks hold an equal obj (e.g. the number
    of work items per d: parts dealt from different item lists would overlap
    or miss pairs without any other error)."""
    if dist is None:
        return
    objs = [None] * dist.get_world_size()
    dist.all_gather_object(objs, obj)
    if any(o != objs[0] for o in objs):
        raise RuntimeError(f"ranks disagree on {what}: {objs}")


# The paper's synthetic sets (Sec. 5.1: i.i.d. exponential, lambda = 40, 2e6
# points) at the largest eps its Table 3 lists for each (Table 2 times
# Syn16D2M at eps = 0.05).
SYN_EPS = {16: 0.05, 32: 0.10, 64: 0.18}


def workload_name(args, runs) -> str:
    if args.workload == "exponential":
        return (f"paper's Syn16/32/64D2M shape: exponential (lambda=40) [0,1]^d, n={args.n}, "
                f"d in {[r['d'] for r in runs]}, eps {[r['eps'] for r in runs]} (Table 3)")
    return (f"paper-scale uniform [0,1)^d, n={args.n}, d in {[r['d'] for r in runs]}, "
            f"eps for 32 mean neighbours")


def workload(args):
    with open(WORKLOADS) as f:
        W = json.load(f)
    dims = [int(x) for x in (args.dims or ("16,32,64" if args.form == "tc" else "16")).split(",")]
    runs = []
    for d in dims:
        if args.workload == "exponential":
            runs.append(dict(d=d, n=args.n, eps=SYN_EPS[d], seed=4000 + d, kind="exponential", depth=None))
            continue
        w = W[f"paper_d{d}"]
        runs.append(dict(d=d, n=args.n, eps=w["eps"], seed=w["seed"], kind="uniform",
                         depth=w.get("depth_per_pair")))
    return runs


def cpu_baseline(runs, budget_s=15.0):
    """The oracle, as it stands, on a bounded sample: the first m points of each
    run's point set, m sized for ~budget_s of CPU work in total."""
    import oracle
    cores = os.cpu_count() or 1
    evals, secs, parts = 0, 0.0, []
    per = budget_s / len(runs)
    for r in runs:
        m = 8000
        while True:
            X = synth.generate(r["kind"], m, r["d"], r["seed"])
            t = time.perf_counter()
            st = oracle.grid_count(X, r["eps"], k=1)
            dt = time.perf_counter() - t
            if dt > per * 0.3 or m >= r["n"]:
                break
            m = min(r["n"], int(m * math.sqrt(per / max(dt, 1e-3)) * 0.9))
        evals += st["candidates"]
        secs += dt
        parts.append(f"first {m} points of the d={r['d']} set")
    # one core, on a small sample of the first set (the oracle's rate per core)
    r = runs[0]
    X1 = synth.generate(r["kind"], 6000, r["d"], r["seed"])
    t = time.perf_counter()
    st1 = oracle.grid_count(X1, r["eps"], k=1, nthreads=1)
    one = st1["candidates"] / (time.perf_counter() - t)
    return {"value": evals / secs, "unit": "distance evals/s", "cores": cores, "kind": "oracle",
            "sample": "; ".join(parts) + f"; {secs:.1f} s of CPU work",
            "value_one_core": one, "one_core_sample": f"first 6000 points of the d={r['d']} set",
            "cpu_model": _cpu_model()}


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def reference_arm(args, runs):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = args.steps if args.steps is not None else 2
    import oracle
    oracle.build()
    cb = None
    vals, walls = [], []
    # each step a bounded sample, sized so that the whole run stays near 2.5 minutes
    budget = args.ref_budget or max(3.0, min(20.0, 150.0 / max(1, args.warmup + steps)))
    for _ in range(args.warmup + steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(runs, budget_s=budget)
        walls.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    v = statistics.median(vals[args.warmup:]) if steps else vals[-1]
    ms_step = 1e3 * statistics.median(walls[args.warmup:] if steps else walls)
    out = {"metric": "distance evals/s (self-join, exact pair set)", "value": v,
           "unit": "distance evals/s", "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
           "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_name(args, runs),
                      "form": "cpu-oracle", "sample": cb["sample"]},
           "cpu_baseline": dict(cb, value=v),
           "e2e": {"value": v, "unit": "distance evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def plain_leg(gj, torch, data, col, fp64_tflops, stream, tune=True, full=False):
    """One plain FP64 join (SHORTC, no tensor cores) of the d=16 set, timed by
    the library's CUDA events, with its FP64-pipe roofline fraction."""
    for r, X, Xd in data:
        if r["d"] != 16:
            continue
        kw = {"k": 0}
        t = None
        if tune:
            tcfg = gj.gj_config_init()
            tcfg.stream = stream.cuda_stream
            t = gj.gj_autotune(Xd, r["eps"], tcfg)
            kw = {"k": t["k"], "query_block": t["query_block"], "tile": t["tile"]}
        with gj.Index(Xd[:50_000], r["eps"], stream=stream.cuda_stream, **kw) as w:
            w.count()                                        # load the kernel
        with gj.Index(Xd, r["eps"], stream=stream.cuda_stream, **kw) as ix:
            info = ix.info()
            st, cnt = gj.gj_self_join(ix.h, col["out"][16])
            if st != gj.GJ_OK:
                raise RuntimeError(f"plain join failed: {gj.gj_status_string(st)}")
            s = ix.stats()
        join_s = s["join_ms"] * 1e-3
        achieved = 3.0 * s["dims"] / join_s / 1e12
        peak = 0.75 * fp64_tflops
        out = {"workload": f"d=16 set, n={r['n']}", "join_s": join_s, "pairs": cnt, "k": info["k"],
               "tuned": {f: t[f] for f in ("k", "query_block", "tile", "trials")} if t else None,
               "evals_per_s": info["candidate_pairs"] / join_s,
               "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                            "frac": achieved / peak, "kernel": "k_join_plain",
                            "peak_source": "FP64 FMA probe measured in this run x 3/4 (DADD+DFMA mix)"}}
        if cnt != col["pairs"].get(16):
            out["mismatch"] = f"plain found {cnt} pairs, tc {col['pairs'].get(16)}"
        if full:
            out["full"] = plain_full(gj, data, col, stream, peak)
        else:
            out["sampled"] = plain_sampled(gj, data, col, stream, peak)
        return out
    return None


def plain_full(gj, data, col, stream, peak):
    """The plain FP64 join of the d = 32 and 64 sets over the whole set, once
    each, into the device buffer the tensor-core form filled: measured join
    time, FP64 roofline fraction, equal |R|, and the join-time ratio."""
    res = {}
    steps = max(1, col.get("steps", 1))
    for r, X, Xd in data:
        if r["d"] == 16:
            continue
        with gj.Index(Xd, r["eps"], k=0, stream=stream.cuda_stream) as ix:
            info = ix.info()
            st, cnt = gj.gj_self_join(ix.h, col["out"][r["d"]])
            if st != gj.GJ_OK:
                raise RuntimeError(f"plain join failed: {gj.gj_status_string(st)}")
            s = ix.stats()
        join_s = s["join_ms"] * 1e-3
        achieved = 3.0 * s["dims"] / join_s / 1e12
        tc_s = col["join_ms_d"].get(r["d"], 0.0) * 1e-3 / steps
        res[r["d"]] = {"join_s": join_s, "pairs": cnt, "k": info["k"],
                       "same_count_as_tc": cnt == col["pairs"].get(r["d"]),
                       "evals_per_s": info["candidate_pairs"] / join_s, "fp64_frac": achieved / peak,
                       "tc_join_speedup": join_s / tc_s if tc_s else None}
    return res


def plain_sampled(gj, data, col, stream, peak, nparts=32):
    """The plain FP64 join of the d = 32 and 64 sets would take minutes, so it
    runs on one part of an entity partition (Sec. 6.2: load-ordered work items
    dealt round-robin, a load-stratified 1/nparts sample, count only); its
    kernel busy time (each SM's occupied span averaged over the SMs) x
    nparts estimates the whole join, beside the tensor-core form's measured
    join time of the same set."""
    res = {}
    steps = max(1, col.get("steps", 1))
    for r, X, Xd in data:
        if r["d"] == 16:
            continue
        with gj.Index(Xd, r["eps"], k=0, stream=stream.cuda_stream) as ix:
            st, cnt = gj.gj_self_join_part(ix.h, nparts // 2, nparts, None)
            if st != gj.GJ_OK:
                raise RuntimeError(f"plain sampled join failed: {gj.gj_status_string(st)}")
            s = ix.stats()
        est_s = s["busy_ms"] * 1e-3 * nparts
        achieved = 3.0 * s["dims"] / (s["busy_ms"] * 1e-3) / 1e12
        tc_s = col["join_ms_d"].get(r["d"], 0.0) * 1e-3 / steps
        res[r["d"]] = {"part": f"{nparts // 2} of {nparts}", "join_s_est": est_s, "pairs_in_part": cnt,
                       "fp64_frac": achieved / peak,
                       "tc_join_speedup_est": est_s / tc_s if tc_s else None}
    return res


def bench_jobs(args):
    """The many-jobs workload: 256 independent self-joins (n log-uniform in
    [1k, 200k], d in {16, 18, 32}, uniform and mixture data alternating, eps per
    job for 8-128 mean neighbours) built and joined in one persistent,
    graph-captured launch.  Step = gj_batch_build + gj_batch_self_join."""
    import torch
    from paper_1809_09930_gb300 import gj
    with open(WORKLOADS) as f:
        specs = json.load(f)["jobs"]
    steps = args.steps if args.steps is not None else 5
    stream = torch.cuda.current_stream()
    jobs = []
    for js in specs:
        X = synth.generate(js["kind"], js["n"], js["d"], js["seed"])
        jobs.append((torch.from_numpy(X).cuda(), js["eps"], 0))
    torch.cuda.synchronize()
    cfg = gj.gj_config_init()
    cfg.stream = stream.cuda_stream
    if not args.no_tune:
        cfg.flags = gj.GJ_DEFAULT_FLAGS | gj.GJ_AUTOTUNE
    # the first build runs the autotuner's trials (per-job k); later builds of
    # the same job list reuse its picks
    t0 = time.perf_counter()
    b = gj.gj_batch_build(jobs, cfg)
    tune_s = time.perf_counter() - t0
    ks = gj.gj_batch_get_k(b, len(jobs))
    info = gj.gj_batch_get_info(b)
    # per-job contraction work at the picked k, outside the timing
    flops = 0.0
    for (X, eps, _), js, k in zip(jobs, specs, ks):
        with gj.Index(X, eps, k=k, flags=gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER) as ix:
            flops += 2.0 * js["d"] * ix.info()["candidate_pairs"]
    st, counts = gj.gj_batch_self_join(b, len(jobs))
    outs = [torch.empty((c + 16, 2), dtype=torch.int32, device="cuda") for c in counts]
    gj.gj_batch_free(b)

    def step():
        bb = gj.gj_batch_build(jobs, cfg)
        st, c = gj.gj_batch_self_join(bb, len(jobs), outs)
        if st != gj.GJ_OK or c != counts:
            raise RuntimeError(f"batch join: {gj.gj_status_string(st)}")
        return bb

    for _ in range(args.warmup):
        gj.gj_batch_free(step())
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    l0 = gj.gj_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    handles = []
    for _ in range(steps):
        handles.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = gj.gj_kernel_launches() - l0
    ms = ev0.elapsed_time(ev1)
    # the join alone: replay of the captured graph on the last batch
    bb = handles[-1]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        gj.gj_batch_self_join(bb, len(jobs), outs)
    e1.record(stream)
    torch.cuda.synchronize()
    join_ms = e0.elapsed_time(e1) / reps
    for h in handles:
        gj.gj_batch_free(h)
    with open(PEAKS) as f:
        pk = json.load(f)
    peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
    achieved = flops / (join_ms * 1e-3) / 1e12
    evals = info["candidate_pairs"]
    out = {
        "metric": "distance evals/s (self-join, exact pair set)",
        "value": evals * steps / (ms * 1e-3), "unit": "distance evals/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f16xf16->f32 filter + f64 recheck", "data": "synthetic",
        "config": {"workload": f"{len(jobs)} independent self-joins in one launch, {info['total_points']} points",
                   "form": "tc-batch", "work_items": info["work_items"], "pairs": int(sum(counts)),
                   "step": "gj_batch_build (all indices) + gj_batch_self_join (one graph-captured launch)",
                   "k_histogram": {k: ks.count(k) for k in sorted(set(ks))},
                   "first_build_with_tuning_s": tune_s},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_join_tc (many-jobs)",
                     "join_ms_graph_replay": join_ms},
        "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(out), flush=True)


def bench_qe(args):
    """The similarity join Q join_eps E (Sec. 3.1): the 2M-point d = 16 set as
    the entries (index built once, outside the timing), args.nq fresh uniform
    queries; step = gj_join_qe into a device buffer.  Unit: query x entry
    pairs in adjacent cells."""
    import torch
    from paper_1809_09930_gb300 import gj
    with open(WORKLOADS) as f:
        w = json.load(f)["paper_d16"]
    # (the tensor-core join takes ~40 ms: more steps give the clock sampler a
    # second of load)
    steps = args.steps if args.steps is not None else (30 if args.form == "tc" else 3)
    stream = torch.cuda.current_stream()
    E = torch.from_numpy(synth.uniform(args.n, 16, w["seed"])).cuda()
    Qh = synth.uniform(args.nq, 16, w["seed"] + 7919)
    Q = torch.from_numpy(Qh).cuda()
    tc = args.form == "tc"
    flags = gj.GJ_DEFAULT_FLAGS | (gj.GJ_TC_FILTER if tc else 0)
    ix = gj.Index(E, w["eps"], k=0, flags=flags, stream=stream.cuda_stream)
    st, m = gj.gj_join_qe(ix.h, Q, None)
    out = torch.empty((m + 16, 2), dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        gj.gj_join_qe(ix.h, Q, out)
    fp64 = gj.gj_probe_fp64_tflops()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    l0 = gj.gj_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    join_ms, dims, cand, surv = 0.0, 0, 0, 0
    for _ in range(steps):
        st, m2 = gj.gj_join_qe(ix.h, Q, out)
        if st != gj.GJ_OK or m2 != m:
            raise RuntimeError(f"qe join: {gj.gj_status_string(st)}")
        s = ix.stats()
        join_ms += s["join_ms"]
        dims += s["dims"]
        cand += s["candidates"]
        surv += s["tc_survivors"]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = gj.gj_kernel_launches() - l0
    ms = ev0.elapsed_time(ev1)
    # end to end: host queries in, host pairs out (pinned)
    hq = torch.from_numpy(Qh).pin_memory()
    hout = torch.empty((m + 16, 2), dtype=torch.int32).pin_memory()
    t0 = time.perf_counter()
    for _ in range(steps):
        gj.gj_join_qe(ix.h, hq, hout)
    e2e_s = time.perf_counter() - t0
    ix.close()
    if tc:
        # contraction work: 2*d FLOPs per query x entry candidate pair
        with open(PEAKS) as f:
            pk = json.load(f)
        peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
        achieved = 2.0 * 16 * cand / (join_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_join_tc (asymmetric)",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (fp16 runs at the bf16 rate)",
                "join_ms_per_step": join_ms / steps, "survivors_per_step": surv / steps}
    else:
        achieved = 3.0 * dims / (join_ms * 1e-3) / 1e12
        peak = 0.75 * fp64
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_join_plain (asymmetric)",
                "peak_source": "FP64 FMA probe measured in this run x 3/4 (DADD+DFMA mix)",
                "join_ms_per_step": join_ms / steps}
    cb = None
    if not args.no_baseline:
        import oracle
        mq = 2000
        t = time.perf_counter()
        oracle.brute_qe(Qh[:mq], E.cpu().numpy(), w["eps"])
        dt = time.perf_counter() - t
        cb = {"value": mq * args.n / dt, "unit": "distance evals/s", "cores": os.cpu_count(), "kind": "oracle",
              "sample": f"nested loop of the first {mq} queries against all {args.n} entries, {dt:.1f} s"}
    out_line = {
        "metric": "distance evals/s (similarity join Q join_eps E, exact pair set)",
        "value": cand / (ms * 1e-3), "unit": "distance evals/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f16xf16->f32 filter + f64 recheck" if tc else "f64", "data": "synthetic",
        "config": {"workload": f"Q join_eps E: {args.nq} uniform queries x {args.n} uniform entries, d=16, "
                               f"eps {w['eps']}", "form": args.form, "pairs": m,
                   "step": "gj_join_qe (query side build + one join launch) into a device buffer"},
        "roofline": roof,
        "cpu_baseline": cb,
        "e2e": {"value": cand / e2e_s, "unit": "distance evals/s", "h2d_bytes_per_step": int(Qh.nbytes),
                "d2h_bytes_per_step": 8 * m},
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(out_line), flush=True)


def main():
    args = parse()
    if args.workload in ("jobs", "qe") and args.impl == "ours":
        # one-GPU workloads: under torchrun rank 0 runs them, the other ranks exit
        if int(os.environ.get("RANK", "0")) != 0:
            return
        (bench_jobs if args.workload == "jobs" else bench_qe)(args)
        return
    runs = workload(args)
    if args.impl == "reference":
        reference_arm(args, runs)
        return

    import torch
    from paper_1809_09930_gb300 import gj

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    steps = args.steps if args.steps is not None else (1 if args.form == "plain" else 5)
    flags = gj.GJ_DEFAULT_FLAGS | (gj.GJ_TC_FILTER if args.form == "tc" else 0)
    stream = torch.cuda.current_stream()

    # inputs resident in HBM before the timed region; outputs to a device buffer
    data = []
    for r in runs:
        X = synth.generate(r["kind"], r["n"], r["d"], r["seed"])
        Xd = torch.from_numpy(X).to("cuda")
        data.append((r, X, Xd))
    torch.cuda.synchronize()

    # autotuner: k, query block and tile per d by timed trials, once, before
    # the warm-up; every step then builds with the picks
    # (rank 0 tunes; every rank builds with its picks)
    tuned = {}
    tune_s = 0.0
    if not args.no_tune:
        t0 = time.perf_counter()
        if rank == 0:
            for r, X, Xd in data:
                tcfg = gj.gj_config_init()
                tcfg.flags = flags
                tcfg.stream = stream.cuda_stream
                tuned[r["d"]] = gj.gj_autotune(Xd, r["eps"], tcfg)
        tuned = agree(dist, tuned)
        tune_s = time.perf_counter() - t0
    check_same(dist, {d: settings_of(t) for d, t in tuned.items()}, "the tuned settings")

    def settings(d):
        return settings_of(tuned.get(d))

    def one_step(collect):
        tot_evals = 0
        for r, X, Xd in data:
            ix = gj.Index(Xd, r["eps"], flags=flags, stream=stream.cuda_stream, **settings(r["d"]))
            info = ix.info()
            cap = collect["cap"].get(r["d"])
            if cap is None:
                cnt = ix.count()
                cap = int(cnt * 1.02) + 1024
                collect["cap"][r["d"]] = cap
                collect["out"][r["d"]] = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
            st, cnt = gj.gj_self_join_part(ix.h, rank, world, collect["out"][r["d"]])
            if st != gj.GJ_OK:
                raise RuntimeError(f"join failed: {gj.gj_status_string(st)}")
            s = ix.stats()
            collect["join_ms"] += s["join_ms"]
            collect["join_ms_d"][r["d"]] = collect["join_ms_d"].get(r["d"], 0.0) + s["join_ms"]
            collect["launches_join"] += s["launches"]
            collect["dims"] += s["dims"]
            collect["evaluated"] += s["evaluated"]
            collect["pairs"][r["d"]] = cnt
            collect["k"][r["d"]] = info["k"]
            collect["items"][r["d"]] = info["work_items"]
            collect["flops"] += 2.0 * r["d"] * info["candidate_pairs"] / world
            collect["survivors"] += s["tc_survivors"]
            tot_evals += info["candidate_pairs"]
            ix.close()
        return tot_evals

    def fresh():
        return {"cap": {}, "out": {}, "join_ms": 0.0, "launches_join": 0, "dims": 0, "evaluated": 0,
                "pairs": {}, "k": {}, "items": {}, "flops": 0.0, "survivors": 0, "join_ms_d": {}}

    col = fresh()
    for _ in range(args.warmup):
        one_step(col)
    if args.warmup:
        check_same(dist, col["items"], "the work items per d")
    fp64_tflops = gj.gj_probe_fp64_tflops()

    keep = {"cap": col["cap"], "out": col["out"]}
    col = fresh()
    col.update(keep)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = gj.gj_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    evals = 0
    for _ in range(steps):
        evals += one_step(col)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = gj.gj_kernel_launches() - l0
    clk = clocks.stop()
    ms = rank_max(dist, ev0.elapsed_time(ev1))
    if not args.warmup:
        check_same(dist, col["items"], "the work items per d")
    ds = sorted(col["pairs"])
    col["pairs"] = dict(zip(ds, rank_sum(dist, [col["pairs"][d] for d in ds])))
    # evals: the whole job's candidate pairs (parts of one join sum to the join)
    value = evals / (ms * 1e-3)

    # roofline of the dominant kernel (the join), from its own CUDA-event time
    join_s = col["join_ms"] * 1e-3
    if args.form == "plain":
        # FP64 pipe: 2 instructions (DADD, DFMA) = 3 FLOPs per evaluated dimension;
        # the mix's ceiling is 3/4 of the FMA-only rate the probe measures.
        achieved = 3.0 * col["dims"] / join_s / 1e12
        peak = 0.75 * fp64_tflops
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "k_join_plain", "peak_source": "FP64 FMA probe measured in this run x 3/4 "
                "(DADD+DFMA mix)", "fp64_fma_tflops_measured": fp64_tflops}
    else:
        # contraction work: 2*d FLOPs per unordered candidate pair (the dot
        # product a.b; norms and padding excluded) over the join kernels' time
        with open(PEAKS) as f:
            pk = json.load(f)
        peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
        achieved = col["flops"] / join_s / 1e12
        # DRAM traffic of one 2M-point d = 32 launch: the ncu capture of a 1M-point launch of this
        # kernel (3.53 GB: operand re-reads and recheck gathers) scaled by its candidate pairs (x 4)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": 14.1e9 if args.workload == "paper" else None,
                "traffic_note": "bytes per d=32 launch at n=2e6, scaled from a 1e6-point ncu capture",
                "kernel": "k_join_tc",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (fp16 runs at the bf16 rate)",
                "survivors_per_step": col["survivors"] / steps}

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        hin = [torch.from_numpy(X).pin_memory() for _, X, _ in data]
        hout = {r["d"]: torch.empty((col["cap"][r["d"]], 2), dtype=torch.int32).pin_memory()
                for r, _, _ in data}
        phases = {"build_s": 0.0, "join_s": 0.0, "close_s": 0.0}

        def e2e_step():
            ev = 0
            for (r, X, _), hx in zip(data, hin):
                t = tuned.get(r["d"])
                p0 = time.perf_counter()
                ix = gj.Index(hx, r["eps"], flags=flags, batch_pairs=t["batch_pairs"] if t else 0,
                              **settings(r["d"]))
                info = ix.info()
                p1 = time.perf_counter()
                st, cnt = gj.gj_self_join_part(ix.h, rank, world, hout[r["d"]])
                if st != gj.GJ_OK:
                    raise RuntimeError(gj.gj_status_string(st))
                p2 = time.perf_counter()
                ev += info["candidate_pairs"]
                ix.close()
                phases["build_s"] += p1 - p0
                phases["join_s"] += p2 - p1
                phases["close_s"] += time.perf_counter() - p2
            return ev
        e2e_step()
        torch.cuda.synchronize()
        for k in phases:
            phases[k] = 0.0
        t0 = time.perf_counter()
        ev = 0
        for _ in range(steps):
            ev += e2e_step()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = rank_max(dist, e2e_s)
        h2d = sum(X.nbytes for _, X, _ in data)
        d2h = sum(8 * col["pairs"][r["d"]] for r, _, _ in data)
        e2e = {"value": ev / e2e_s, "unit": "distance evals/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "ms_per_step_by_phase": {k.replace("_s", ""): 1e3 * v / steps for k, v in phases.items()}}

    # the plain FP64 form of the same d=16 join, once, for the TC-vs-plain ratio
    plain = None
    if args.form == "tc" and not args.no_plain and rank == 0 and world == 1:
        col["steps"] = steps
        plain = plain_leg(gj, torch, data, col, fp64_tflops, stream, tune=not args.no_tune, full=args.plain_full)
        if plain and col["join_ms_d"].get(16):
            # same join, same exact pair set: join time of the plain form over the tc form's
            plain["tc_join_speedup"] = plain["join_s"] / (col["join_ms_d"][16] * 1e-3 / steps)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cb = None if (args.no_baseline or world > 1) else cpu_baseline(runs)
    out = {
        "metric": "distance evals/s (self-join, exact pair set)",
        "value": value,
        "unit": "distance evals/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": ms / steps,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f64" if args.form == "plain" else "f16xf16->f32 filter + f64 recheck",
        "data": "synthetic",
        "config": {"workload": workload_name(args, runs),
                   "form": args.form, "eps": {r["d"]: r["eps"] for r in runs}, "k": col["k"],
                   "pairs": col["pairs"], "parallelism": f"entity partition x{world}",
                   "l2": "inputs larger than L2 (>=256 MB per point set)",
                   "step": "index build (REORDER, grid, adjacency, queue) + join into a device buffer",
                   "tuned": {d: {f: t[f] for f in ("k", "query_block", "tile", "batch_pairs", "trials")}
                             for d, t in tuned.items()},
                   "tune_s": tune_s},
        "roofline": roof,
        "cpu_baseline": cb,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "join_stats": {"join_ms_total": col["join_ms"], "join_launches": col["launches_join"],
                       "join_ms_per_step_by_d": {d: v / steps for d, v in col["join_ms_d"].items()},
                       "dims_evaluated": col["dims"], "pairs_evaluated": col["evaluated"]},
        "plain_fp64": plain,
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
