"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (index from device-resident points, all flags on, automatic k).

The oracle cannot redo a whole 2e12-pair join in test time, so every check
here is either per sampled query (the oracle's brute-force neighbour list of
that point, `gjo_query_neighbors`, against the GPU's pairs (q, *)) or a
property that holds at any size (symmetry, self-pairs, equality of the plain
and tensor-core forms).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import TIE_REL

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


def _w(name):
    with open(os.path.join(GOLD, "workloads.json")) as f:
        return json.load(f)[name]


def _device_join(X, eps, flags, k=0):
    Xd = torch.from_numpy(X).cuda()
    with gj.Index(Xd, eps, k=k, flags=flags) as ix:
        n = ix.count()
        out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        st, m = gj.gj_self_join(ix.h, out)
        assert st == gj.GJ_OK and m == n
        info = ix.info()
    keys = (out[:, 0].to(torch.int64) << 32) | (out[:, 1].to(torch.int64) & 0xFFFFFFFF)
    keys = torch.sort(keys).values
    return keys, info


def _check_queries(X, eps, keys_sorted: torch.Tensor, queries):
    """GPU neighbours of each sampled query = the oracle's brute-force list, up to ties."""
    e2 = eps * eps
    ks = keys_sorted
    for q in queries:
        lo = int(torch.searchsorted(ks, torch.tensor([q << 32], device=ks.device)).item())
        hi = int(torch.searchsorted(ks, torch.tensor([(q + 1) << 32], device=ks.device)).item())
        got = (ks[lo:hi] & 0xFFFFFFFF).cpu().numpy().astype(np.uint32)
        ref = oracle.query_neighbors(X, eps, int(q))
        for j in np.setxor1d(got, ref):
            s = oracle.sqdist(X[q], X[int(j)])
            assert abs(s - e2) <= TIE_REL * e2, f"query {q}: neighbour {j} differs (s={s}, e2={e2})"


def _check_properties(keys_sorted: torch.Tensor, n: int):
    a = keys_sorted >> 32
    b = keys_sorted & 0xFFFFFFFF
    assert int((a == b).sum().item()) == n                         # every self-pair, once
    assert bool((keys_sorted[1:] != keys_sorted[:-1]).all().item())  # no duplicates
    sym = torch.sort((b << 32) | a).values                          # (a,b) in R <=> (b,a) in R
    assert torch.equal(sym, keys_sorted)


def _queries(n, seed, m=48):
    return sorted(set((synth.uniform01(seed, m) * n).astype(np.int64).tolist()))


@pytest.mark.parametrize("name", ["paper_d16", "paper_d32", "paper_d64"])
def test_paper_scale_tc(name):
    w = _w(name)
    X = synth.uniform(w["n"], w["d"], w["seed"])
    keys, info = _device_join(X, w["eps"], TC)
    assert info["candidate_pairs"] == w["n"] * (w["n"] - 1) // 2
    _check_properties(keys, w["n"])
    _check_queries(X, w["eps"], keys, _queries(w["n"], 7 + w["d"]))
    # S_D close to the 32 mean neighbours the workload's eps was chosen for
    sd = oracle.selectivity(keys.numel(), w["n"])
    assert 24 < sd < 42


def test_paper_scale_d16_plain_equals_tc_count():
    w = _w("paper_d16")
    X = torch.from_numpy(synth.uniform(w["n"], w["d"], w["seed"])).cuda()
    with gj.Index(X, w["eps"], k=0) as ip:
        n_plain = ip.count()
    with gj.Index(X, w["eps"], k=0, flags=TC) as it:
        n_tc = it.count()
    assert n_plain == n_tc


@pytest.mark.parametrize("flags", [gj.GJ_DEFAULT_FLAGS, TC])
def test_mixture_d90(flags):
    w = _w("mixture_d90")
    X = synth.mixture(w["n"], w["d"], w["seed"])
    keys, info = _device_join(X, w["eps"], flags)
    _check_properties(keys, w["n"])
    _check_queries(X, w["eps"], keys, _queries(w["n"], 90, m=40))


def test_large_skewed_streamed_to_pinned_host():
    """5M x 18 skewed set: the result (~3e8 pairs) is emitted in result batches
    (b_s = 1e8 when the estimate exceeds 3e8, Sec. 3.2.2) and streamed to
    pinned host memory while the next batch runs (GJ_HOST_BATCHED: without it
    the kernels would write the pinned buffer directly)."""
    w = _w("skewed")
    X = synth.skewed(w["n"], w["d"], w["seed"])
    Xd = torch.from_numpy(X).cuda()
    with gj.Index(Xd, w["eps"], k=0, flags=TC | gj.GJ_HOST_BATCHED) as ix:
        n = ix.count()
        host = torch.empty((n, 2), dtype=torch.int32).pin_memory()
        st, m = gj.gj_self_join(ix.h, host)
        stats = ix.stats()
    assert st == gj.GJ_OK and m == n
    assert stats["estimate"] > 300_000_000 and stats["batch_pairs"] == 100_000_000
    assert stats["launches"] >= stats["batches_planned"] >= 3
    t = host.cuda()
    keys = torch.sort((t[:, 0].to(torch.int64) << 32) | (t[:, 1].to(torch.int64) & 0xFFFFFFFF)).values
    del t
    _check_properties(keys, w["n"])
    _check_queries(X, w["eps"], keys, _queries(w["n"], 55, m=32))


def test_paper_syn16d2m_tc_sampled_queries():
    """The paper's own Syn16D2M shape (Sec. 5.1: 2e6 exponential points,
    lambda = 40, in 16-D) at eps = 0.05 (Table 2): dense co-located data, |R|
    about 2.4e9.  The result stays on the device; each sampled query's list is
    selected by a scan (no sort of the whole result)."""
    n, d, eps = 2_000_000, 16, 0.05
    X = synth.exponential(n, d, 4016)
    Xd = torch.from_numpy(X).cuda()
    with gj.Index(Xd, eps, k=0, flags=TC) as ix:
        m = ix.count()
        out = torch.empty((m, 2), dtype=torch.int32, device="cuda")
        st, m2 = gj.gj_self_join(ix.h, out)
    assert st == gj.GJ_OK and m2 == m
    assert int((out[:, 0] == out[:, 1]).sum().item()) == n
    e2 = eps * eps
    for q in _queries(n, 16, m=24):
        sel = out[:, 0] == q
        got = np.sort(out[sel][:, 1].cpu().numpy().view(np.uint32))
        ref = oracle.query_neighbors(X, eps, int(q))
        for j in np.setxor1d(got, ref):
            s = oracle.sqdist(X[q], X[int(j)])
            assert abs(s - e2) <= TIE_REL * e2, f"query {q}: neighbour {j} differs"
        # the reverse orientation of every listed pair is present too
        rev = int(((out[:, 1] == q)).sum().item())
        assert rev == got.size


def test_large_skewed_plain_equals_tc_count():
    """The 5M x 18 skewed set in both forms: the plain FP64 join and the
    tensor-core filtered join count the same |R|."""
    w = _w("skewed")
    X = torch.from_numpy(synth.skewed(w["n"], w["d"], w["seed"])).cuda()
    with gj.Index(X, w["eps"], k=0) as ip:
        n_plain = ip.count()
    with gj.Index(X, w["eps"], k=0, flags=TC) as it:
        n_tc = it.count()
    assert n_plain == n_tc > 300_000_000


def _device_keys(out: torch.Tensor, m: int) -> torch.Tensor:
    t = out[:m]
    return torch.sort((t[:, 0].to(torch.int64) << 32) | (t[:, 1].to(torch.int64) & 0xFFFFFFFF)).values


@pytest.mark.parametrize("name", ["paper_d32", "paper_d64"])
def test_paper_scale_plain_fp64_full(name):
    """The plain FP64 form (SHORTC, no tensor cores) over the whole 2M-point set
    at d = 32 and 64, once (about 1.5 and 4 minutes): the same pair set as the
    tensor-core form, bit for bit, and the oracle's list for sampled queries."""
    w = _w(name)
    X = synth.uniform(w["n"], w["d"], w["seed"])
    Xd = torch.from_numpy(X).cuda()
    with gj.Index(Xd, w["eps"], k=0, flags=TC) as it:
        n = it.count()
        out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        st, m = gj.gj_self_join(it.h, out)
        assert st == gj.GJ_OK and m == n
    tc_keys = _device_keys(out, n)
    with gj.Index(Xd, w["eps"], k=0) as ip:
        st, m = gj.gj_self_join(ip.h, out)           # the tensor-core count sizes the buffer
        assert st == gj.GJ_OK and m == n
        s = ip.stats()
    print(f"{name}: plain FP64 join {s['join_ms'] / 1e3:.1f} s, |R| = {n}")
    plain_keys = _device_keys(out, n)
    assert torch.equal(plain_keys, tc_keys)
    _check_properties(plain_keys, w["n"])
    _check_queries(X, w["eps"], plain_keys, _queries(w["n"], 11 + w["d"], m=24))


def test_mixture_d32_tc_against_the_oracle():
    """The 68,000 x 32 mixture (stands in for ColorHist/LayoutHist, Table 1) in
    the tensor-core form at its full size, element by element against the
    oracle's grid join."""
    from tests.parity import assert_parity
    w = _w("mixture_d32")
    X = synth.mixture(w["n"], w["d"], w["seed"])
    keys, info = _device_join(X, w["eps"], TC)
    _check_properties(keys, w["n"])
    got = np.stack([(keys >> 32).cpu().numpy(), (keys & 0xFFFFFFFF).cpu().numpy()], axis=1).astype(np.uint32)
    assert_parity(X, w["eps"], got, oracle.grid_join(X, w["eps"], 3))


def test_many_jobs_full_size():
    """The full many-jobs workload (256 jobs, n log-uniform in [1k, 200k], 10 M
    points, d in {16, 18, 32}, uniform and mixture alternating, eps per job for
    8-128 mean neighbours) in one graph-captured launch: every job's pairs equal
    its own single join, a replay of the graph gives the same pairs, and the 8
    largest jobs match the oracle on sampled queries."""
    with open(os.path.join(GOLD, "workloads.json")) as f:
        specs = json.load(f)["jobs"]
    assert len(specs) == 256
    data = [synth.generate(js["kind"], js["n"], js["d"], js["seed"]) for js in specs]
    jobs = [(torch.from_numpy(X).cuda(), js["eps"], 0) for X, js in zip(data, specs)]
    b = gj.gj_batch_build(jobs)
    try:
        st, counts = gj.gj_batch_self_join(b, len(jobs))
        assert st == gj.GJ_OK
        outs = [torch.empty((c + 8, 2), dtype=torch.int32, device="cuda") for c in counts]
        st, c1 = gj.gj_batch_self_join(b, len(jobs), outs)
        assert st == gj.GJ_OK and c1 == counts
        first = [_device_keys(o, c) for o, c in zip(outs, counts)]
        st, c2 = gj.gj_batch_self_join(b, len(jobs), outs)          # graph replay
        assert st == gj.GJ_OK and c2 == counts
        for j, (o, c) in enumerate(zip(outs, counts)):
            assert torch.equal(_device_keys(o, c), first[j]), f"replay differs on job {j}"
    finally:
        gj.gj_batch_free(b)
    for j, (Xd, eps, _) in enumerate(jobs):
        with gj.Index(Xd, eps, k=0, flags=TC) as ix:
            n = ix.count()
            assert n == counts[j], f"job {j}"
            single = torch.empty((n, 2), dtype=torch.int32, device="cuda")
            st, m = gj.gj_self_join(ix.h, single)
            assert st == gj.GJ_OK and m == n
        assert torch.equal(_device_keys(single, n), first[j]), f"job {j} differs from its single join"
    largest = sorted(range(len(specs)), key=lambda j: -specs[j]["n"])[:8]
    for j in largest:
        _check_properties(first[j], specs[j]["n"])
        _check_queries(data[j], specs[j]["eps"], first[j], _queries(specs[j]["n"], 300 + j, m=12))
