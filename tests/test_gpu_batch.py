"""Many independent self-joins in one persistent, graph-captured launch.

Every job's pairs from the combined launch must equal that job's own
tensor-core join exactly (the combined layout only pads dimensions with zeros,
which add exactly 0 to an FP64 sum), and agree with the oracle up to the tie
band; a second call replays the captured graph and must give the same result.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import assert_parity, keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")

TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


def _jobs(count, seed, n_hi):
    out = []
    for js in synth.many_jobs(count=count, seed=seed, n_lo=300, n_hi=n_hi):
        X = synth.generate(js.kind, js.n, js.d, js.seed)
        # eps for roughly the job's target neighbour count: scale a unit-cube guess
        m = min(js.n, 1500)
        lo, hi = 1e-3, 3.0
        for _ in range(18):
            mid = (lo * hi) ** 0.5
            sd = (oracle.brute_count(X[:m], mid) - m) / m
            if sd < js.target_nb * (m - 1) / max(js.n - 1, 1):
                lo = mid
            else:
                hi = mid
        out.append((X, (lo * hi) ** 0.5, 0))
    return out


def _single(X, eps):
    with gj.Index(X, eps, k=0, flags=TC) as ix:
        return keys(ix.join())


def test_batch_equals_single_jobs_and_replays():
    jobs = _jobs(24, 7, 12_000)
    b = gj.gj_batch_build(jobs)
    try:
        info = gj.gj_batch_get_info(b)
        assert info["total_points"] == sum(len(X) for X, _, _ in jobs)
        st, counts = gj.gj_batch_self_join(b, len(jobs))           # count only
        assert st == gj.GJ_OK
        outs = [torch.full((c + 8, 2), -1, dtype=torch.int32, device="cuda") for c in counts]
        for rep in range(2):                                         # capture, then replay
            st, counts2 = gj.gj_batch_self_join(b, len(jobs), outs)
            assert st == gj.GJ_OK and counts2 == counts
            for j, (X, eps, _) in enumerate(jobs):
                got = keys(outs[j][:counts[j]].cpu().numpy().view(np.uint32))
                assert np.array_equal(got, _single(X, eps)), f"job {j}"
                assert int(outs[j][counts[j]:].min().item()) == -1
        for j in (0, 5, 11):
            X, eps, _ = jobs[j]
            got = outs[j][:counts[j]].cpu().numpy().view(np.uint32)
            assert_parity(X, eps, got, oracle.brute(X, eps))
    finally:
        gj.gj_batch_free(b)


def test_batch_capacity_and_empty_jobs():
    jobs = _jobs(6, 9, 4000)
    jobs.append((np.zeros((0, 16)), 0.5, 0))                       # an empty job
    jobs.append((np.full((50, 18), 0.3), 0.01, 0))                  # all duplicates
    b = gj.gj_batch_build(jobs)
    try:
        st, counts = gj.gj_batch_self_join(b, len(jobs))
        assert counts[-2] == 0 and counts[-1] == 2500
        outs = [torch.empty((max(c // 2, 1), 2), dtype=torch.int32, device="cuda") for c in counts]
        st, c2 = gj.gj_batch_self_join(b, len(jobs), outs)
        assert st == gj.GJ_ERR_CAPACITY and c2 == counts
    finally:
        gj.gj_batch_free(b)
