"""Write tests/golden/workloads.json: the seeded synthetic workloads, with the
search distance ε of each chosen by bisection on oracle neighbour counts.

Run:  python -m oracle.choose_eps            (a few minutes on 8 cores)

Only the oracle counts pairs here; the CUDA library is not involved.  Each ε is
picked on a seeded sample (the first m rows, which are i.i.d. draws like the
rest) so that the mean neighbour count S_D = (|R| − |D|)/|D| of Sec. 5.2 scaled
from the sample to the full n meets the workload's target:
    target_on_sample = target × (m − 1)/(n − 1).
The file also records the SHORTC depth per candidate pair (Sec. 4.4) that the
throughput figures are measured against, estimated from sampled queries over
the full point set, and the oracle's candidate-pair count of the paper's grid.
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

import oracle
import synth

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "tests", "golden", "workloads.json")


def sample_count(Xs: np.ndarray, eps: float) -> float:
    """Mean neighbours (self excluded) of the sample at ε."""
    m, d = Xs.shape
    if m <= 25_000:
        R = oracle.brute_count(Xs, eps)
    else:
        R = oracle.grid_count(Xs, eps, k=min(d, 4))["R"]
    return (R - m) / m


def bisect_eps(Xs: np.ndarray, target: float, lo: float = 1e-4, hi: float = None,
               steps: int = 40, rel: float = 1e-4) -> float:
    d = Xs.shape[1]
    if hi is None:
        span = float(np.max(np.ptp(Xs, axis=0)))
        hi = span * math.sqrt(d)
    for _ in range(steps):
        mid = math.sqrt(lo * hi)
        if sample_count(Xs, mid) < target:
            lo = mid
        else:
            hi = mid
        if hi / lo - 1.0 < rel:
            break
    return round(math.sqrt(lo * hi), 6)


def depth_per_pair(X: np.ndarray, eps: float, nq: int, seed: int) -> float:
    n = X.shape[0]
    perm = oracle.reorder_perm(X)
    qs = (synth.uniform01(synth.derive_seed(seed, 99), nq) * n).astype(np.int64)
    ds, pc = oracle.depth_stats(X, eps, perm, qs)
    return ds / pc


def main(argv=None):
    argv = argv if argv is not None else sys.argv[1:]
    quick = "--quick" in argv
    W = {}

    W["tiny"] = dict(kind="uniform", n=20_000, d=16, seed=1, eps=0.70, k=6,
                     note="eps fixed at 0.70 by the workload definition")
    X = synth.uniform(20_000, 16, 1)
    st = oracle.grid_count(X, 0.70, 6)
    W["tiny"].update(R=st["R"], candidates=st["candidates"],
                     S_D=oracle.selectivity(st["R"], 20_000))
    print("tiny", W["tiny"], flush=True)

    for d in (16, 32, 64):
        n, seed = 2_000_000, 200 + d
        m = 20_000
        Xs = synth.uniform(m, d, seed)      # first m rows of the full set
        eps = bisect_eps(Xs, 32.0 * (m - 1) / (n - 1))
        entry = dict(kind="uniform", n=n, d=d, seed=seed, eps=eps, target_nb=32.0)
        if not quick:
            Xf = synth.uniform(n, d, seed)
            entry["depth_per_pair"] = depth_per_pair(Xf, eps, 64, seed)
            entry["candidates"] = n * (n - 1) // 2   # grid degenerates at this ε (checked in tests)
        W[f"paper_d{d}"] = entry
        print(f"paper_d{d}", entry, flush=True)

    for n, d, seed in ((68_000, 32, 332), (515_000, 90, 390)):
        m = min(n, 20_000)
        Xs = synth.mixture(n, d, seed)[:m]
        eps = bisect_eps(Xs, 64.0 * (m - 1) / (n - 1))
        W[f"mixture_d{d}"] = dict(kind="mixture", n=n, d=d, seed=seed, eps=eps, target_nb=64.0)
        print(f"mixture_d{d}", W[f"mixture_d{d}"], flush=True)

    n, d, seed = 5_000_000, 18, 5
    m = 100_000
    Xs = synth.skewed(n, d, seed)[:m]
    eps = bisect_eps(Xs, 64.0 * (m - 1) / (n - 1), hi=2.0)
    W["skewed"] = dict(kind="skewed", n=n, d=d, seed=seed, eps=eps, target_nb=64.0)
    print("skewed", W["skewed"], flush=True)

    jobs = []
    for j, js in enumerate(synth.many_jobs()):
        m = min(js.n, 2_000)
        Xs = synth.generate(js.kind, js.n, js.d, js.seed)[:m]
        eps = bisect_eps(Xs, js.target_nb * (m - 1) / (js.n - 1), steps=24, rel=1e-3)
        jobs.append(dict(kind=js.kind, n=js.n, d=js.d, seed=js.seed, eps=eps,
                         target_nb=round(js.target_nb, 4)))
    W["jobs"] = jobs
    print("jobs", len(jobs), "points", sum(j["n"] for j in jobs), flush=True)

    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump(W, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
