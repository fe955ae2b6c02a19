"""The multi-rank path on the CPU: two gloo ranks.

Entity partitioning (Sec. 6.2) needs no exchange of data; the ranks only
agree on the step time (the slowest rank) and add up their parts' pair
counts, and they build with one set of autotuner picks (rank 0's, broadcast).
These tests run the bench's own reduction and agreement helpers across two gloo
processes, check the oracle's view of the partition (parts of the query
blocks dealt round-robin are disjoint and their union is R), and check that
the reference arm runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.rank_max(dist, 10.0 + 5.0 * rank, device="cpu")
    counts = bench.rank_sum(dist, [100 + rank, 7 * rank], device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, counts))


def test_rank_reductions_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, counts in res:
        assert ms == 15.0
        assert counts == [201, 7]


def _part_pairs(X, eps, k, part, nparts):
    """R restricted to the query blocks of one part: the oracle's grid, blocks
    of 120 points per cell in cell order, load order = descending
    (block size x points in the searched cells), dealt round-robin; each block
    emits its pairs (i, j >= i) in both orientations."""
    import oracle
    n, d = X.shape
    perm = oracle.reorder_perm(X)
    Y = X[:, perm[:k]]
    width = eps * (1 + 2.0 ** -30)
    coords = oracle.cell_coords(Y, k, Y.min(axis=0), width)
    ncells = coords.max(axis=0) + 1
    ids = np.array([oracle.linearise(c, ncells) for c in coords])
    order = np.argsort(ids, kind="stable")
    uniq, starts = np.unique(ids[order], return_index=True)
    ends = np.append(starts[1:], n)
    blocks = []
    for ci, (s0, e0) in enumerate(zip(starts, ends)):
        nb = oracle.adjacent_nonempty(uniq, coords[order[s0]], ncells)
        pts = sum(ends[np.searchsorted(uniq, b)] - starts[np.searchsorted(uniq, b)] for b in nb)
        for q0 in range(s0, e0, 120):
            blocks.append((-(min(120, e0 - q0)) * pts, ci, q0, min(e0, q0 + 120)))
    blocks.sort(key=lambda b: (b[0], b[1], b[2]))
    e2 = eps * eps
    out = set()
    for r, (_, ci, q0, q1) in enumerate(blocks):
        if r % nparts != part:
            continue
        nb = oracle.adjacent_nonempty(uniq, coords[order[q0]], ncells)
        cand = []
        for b in nb:
            bi = np.searchsorted(uniq, b)
            if b >= uniq[ci]:
                cand.extend(range(starts[bi], ends[bi]))
        for qi in range(q0, q1):
            i = order[qi]
            for cj in cand:
                if cj < qi:
                    continue
                j = order[cj]
                if oracle.sqdist(X[i], X[j]) <= e2:
                    out.add((i, j))
                    out.add((j, i))
    return out


def _pick_worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank's own (timing-based) pick differs; the helper hands every rank rank 0's
    own = {16: {"k": 4 + 3 * rank, "query_block": 120 - 56 * rank, "tile": 64, "batch_pairs": 0,
                "trials": 12}}
    picked = bench.agree(dist, own)
    bench.check_same(dist, {d: bench.settings_of(t) for d, t in picked.items()}, "the tuned settings")
    # ranks whose item lists differ must fail loudly, on every rank
    try:
        bench.check_same(dist, {16: 1000 + rank}, "the work items per d")
        raised = False
    except RuntimeError:
        raised = True
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, picked, raised))


def test_ranks_build_with_rank0_picks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_pick_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((r for r in (q.get(timeout=120) for _ in ps)), key=lambda x: x[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, picked, raised in res:
        assert picked == {16: {"k": 4, "query_block": 120, "tile": 64, "batch_pairs": 0, "trials": 12}}
        assert raised


def test_entity_partition_parts_are_disjoint_and_cover_R():
    import oracle
    import synth
    X = synth.generate("mixture", 700, 3, 11)
    eps = 0.08
    ref = {tuple(p) for p in oracle.brute(X, eps).tolist()}
    parts = [_part_pairs(X, eps, 2, p, 3) for p in range(3)]
    assert set().union(*parts) == ref
    assert sum(len(p) for p in parts) == len(ref)


def test_reference_arm_only_on_rank0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """Rank 0 of the reference arm times the oracle on the host cores and
    prints one JSON line with the contract's keys (no GPU needed)."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-budget", "1.5"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["steps"] == 1 and out["warmup"] == 0 and out["n_gpus"] == 1
    assert out["metric"].startswith("distance evals/s") and out["unit"] == "distance evals/s"
    assert out["e2e"]["value"] == out["value"] and out["e2e"]["h2d_bytes_per_step"] == 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    assert out["config"]["workload"]
