"""GPU parity: the CUDA self-join against the CPU oracle, through the C ABI.

Sizes span several query blocks (128 points) and candidate tiles with ragged
tails; the last tests run the paper-scale configurations on sampled queries.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import assert_parity, keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _join(X, eps, k=0, flags=None, **kw):
    flags = gj.GJ_DEFAULT_FLAGS if flags is None else flags
    with gj.Index(X, eps, k=k, flags=flags, **kw) as ix:
        p = ix.join()
        return p, ix.info(), ix.stats()


def test_tiny_config_against_nested_loop():
    """Tiny workload: 20,000 uniform points in 16-D, eps = 0.70, k = 6."""
    X = synth.uniform(20_000, 16, 1)
    ref = oracle.brute(X, 0.70)
    got, info, st = _join(X, 0.70, k=6)
    res = assert_parity(X, 0.70, got, ref)
    assert info["k"] == 6
    assert st["pairs"] == len(got)
    print("tiny", {k: v for k, v in res.items() if k not in ("ties", "bad")}, "ties", len(res["ties"]))


@pytest.mark.parametrize("kind,n,d,eps,k", [
    ("uniform", 1537, 3, 0.08, 2),
    ("uniform", 3001, 16, 0.9, 4),
    ("uniform", 2049, 33, 1.25, 5),
    ("mixture", 4100, 32, 0.33, 6),
    ("skewed", 6000, 18, 0.12, 6),
    ("exponential", 3000, 16, 0.06, 6),
    ("mixture", 1300, 90, 0.55, 8),
    ("uniform", 700, 64, 2.0, 3),
])
def test_shapes_against_oracle(kind, n, d, eps, k):
    X = synth.generate(kind, n, d, seed=n * 7 + d)
    ref = oracle.grid_join(X, eps, min(k, d))
    got, info, _ = _join(X, eps, k=k)
    assert_parity(X, eps, got, ref)


@pytest.mark.parametrize("flags", [0, gj.GJ_REORDER, gj.GJ_SORTIDU, gj.GJ_SHORTC,
                                   gj.GJ_REORDER | gj.GJ_SORTIDU])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_flags_do_not_change_result(flags, k):
    X = synth.skewed(3000, 18, 2)
    ref = oracle.brute(X, 0.15)
    got, _, _ = _join(X, 0.15, k=k, flags=flags)
    assert_parity(X, 0.15, got, ref)


def test_lattice_exact_no_ties():
    X = synth.lattice(2500, 6, seed=3, side=5)
    for eps in (1.0, math.sqrt(2.0), 2.0):
        ref = oracle.brute(X, eps)
        got, _, _ = _join(X, eps, k=3)
        assert np.array_equal(keys(got), keys(ref))


def test_edge_cases():
    # one point
    got, _, _ = _join(np.zeros((1, 4)), 0.5, k=2)
    assert got.tolist() == [[0, 0]]
    # all duplicates: every ordered pair
    X = np.full((300, 5), 0.5)
    got, _, _ = _join(X, 1e-6, k=3)
    assert len(got) == 300 * 300
    # eps larger than the data: all pairs
    X = synth.uniform(500, 4, 9)
    got, _, _ = _join(X, 10.0, k=2)
    assert len(got) == 500 * 500
    # tiny eps: only self-pairs
    got, _, _ = _join(X, 1e-9, k=4)
    assert len(got) == 500
    # d = 1
    X = synth.uniform(4000, 1, 5)
    ref = oracle.brute(X, 0.001)
    got, _, _ = _join(X, 0.001, k=1)
    assert_parity(X, 0.001, got, ref)


def test_empty_input():
    with gj.Index(np.zeros((0, 3)), 0.5, k=1) as ix:
        assert ix.count() == 0


def test_invalid_arguments():
    X = synth.uniform(10, 3, 1)
    for eps in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(gj.GJError) as e:
            gj.Index(X, eps)
        assert e.value.status == gj.GJ_ERR_INVALID_ARG
    with pytest.raises(gj.GJError) as e:
        gj.Index(X, 0.1, k=4)
    assert e.value.status == gj.GJ_ERR_INVALID_ARG
    Y = X.copy()
    Y[3, 1] = np.nan
    with pytest.raises(gj.GJError) as e:
        gj.Index(Y, 0.1)
    assert e.value.status == gj.GJ_ERR_NONFINITE
    Y[3, 1] = np.inf
    with pytest.raises(gj.GJError) as e:
        gj.Index(Y, 0.1)
    assert e.value.status == gj.GJ_ERR_NONFINITE


def test_capacity_and_count_only():
    X = synth.mixture(3000, 16, 4)
    ref = oracle.brute(X, 0.3)
    with gj.Index(X, 0.3, k=4) as ix:
        assert ix.count() == len(ref)
        small = np.empty((len(ref) // 3, 2), dtype=np.uint32)
        st, n = gj.gj_self_join(ix.h, small)
        assert st == gj.GJ_ERR_CAPACITY and n == len(ref)


def test_small_batches_resume_exactly():
    """A batch buffer far smaller than |R| forces many launches with deferred
    work items; the union must still be exact (Sec. 3.2.2 batching)."""
    X = synth.mixture(6000, 18, 6)
    ref = oracle.brute(X, 0.35)
    with gj.Index(X, 0.35, k=4, batch_pairs=70_000) as ix:
        got = ix.join()
        st = ix.stats()
    assert st["launches"] > 3
    assert_parity(X, 0.35, got, ref)


def test_device_output_buffer():
    torch = pytest.importorskip("torch")
    X = synth.uniform(5000, 16, 12)
    ref = oracle.brute(X, 0.85)
    with gj.Index(X, 0.85, k=4) as ix:
        n = ix.count()
        out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        st, m = gj.gj_self_join(ix.h, out)
        assert st == gj.GJ_OK and m == n
        got = out.cpu().numpy().view(np.uint32)
    assert_parity(X, 0.85, got, ref)


@pytest.mark.parametrize("form", ["plain", "tc"])
def test_pinned_host_output_direct_and_batched(form):
    """Pinned host output is filled by copies.  A tensor-core index joins in
    one pass into a device buffer that is then copied; the plain form, and
    GJ_HOST_BATCHED, go through the result batches of Sec. 3.2.2.  All give R,
    none writes past |R|, and a buffer that is too small gives GJ_ERR_CAPACITY
    with |R|."""
    torch = pytest.importorskip("torch")
    X = synth.mixture(6000, 18, 6)
    ref = oracle.brute(X, 0.35)
    base = gj.GJ_DEFAULT_FLAGS | (gj.GJ_TC_FILTER if form == "tc" else 0)
    for flags, one_pass in ((base, form == "tc"), (base | gj.GJ_HOST_BATCHED, False)):
        with gj.Index(X, 0.35, k=4, flags=flags, batch_pairs=70_000) as ix:
            n = ix.count()
            assert n == len(ref)
            host = torch.full((n + 8, 2), -1, dtype=torch.int32).pin_memory()
            st, m = gj.gj_self_join(ix.h, host)
            stats = ix.stats()
            assert st == gj.GJ_OK and m == n
            if one_pass:
                assert stats["launches"] == 1 and stats["batch_pairs"] == 0
            else:
                assert stats["launches"] > 3 and stats["batch_pairs"] == 70_000
            assert int(host[n:].min()) == -1
            assert_parity(X, 0.35, host[:n].numpy().view(np.uint32), ref)
            small = torch.empty((n // 3, 2), dtype=torch.int32).pin_memory()
            st, m2 = gj.gj_self_join(ix.h, small)
            assert st == gj.GJ_ERR_CAPACITY and m2 == n


def test_device_input_points():
    torch = pytest.importorskip("torch")
    X = synth.skewed(4000, 18, 8)
    ref = oracle.brute(X, 0.14)
    Xd = torch.from_numpy(X).cuda()
    with gj.Index(Xd, 0.14, k=5) as ix:
        got = ix.join()
    assert_parity(X, 0.14, got, ref)


def test_entity_partitions_union_is_exact():
    """Sec. 6.2 entity partitioning: query blocks dealt round-robin to N_b sets."""
    X = synth.uniform(9000, 16, 13)
    ref = oracle.brute(X, 0.95)
    with gj.Index(X, 0.95, k=3) as ix:
        parts = [ix.join(part=p, nparts=4) for p in range(4)]
    allp = np.concatenate(parts)
    assert len(np.unique(keys(allp))) == len(allp)   # disjoint
    assert_parity(X, 0.95, allp, ref)


def test_reorder_perm_and_candidates_match_oracle():
    X = synth.mixture(5000, 32, 21)
    _, info, _ = _join(X, 0.4, k=4)
    perm = oracle.reorder_perm(X)
    _, var = oracle.variance(X)
    # compare where variances are separated (ties may legitimately order either way)
    sv = var[perm]
    for j in range(len(perm) - 1):
        if sv[j] - sv[j + 1] > 1e-12 * sv[j]:
            assert info["perm"][j] == perm[j]
    st = oracle.grid_count(X, 0.4, 4)
    assert info["candidate_pairs"] == st["candidates"]


def test_stats_count_the_shortc_work():
    X = synth.uniform(4000, 16, 31)
    with gj.Index(X, 0.6, k=1, flags=gj.GJ_REORDER | gj.GJ_SHORTC) as ix:
        ix.count()
        st = ix.stats()
    # without SORTIDU every unordered candidate pair (and the self-pairs) is evaluated
    assert st["evaluated"] == 4000 * 3999 // 2 + 4000
    assert st["dims"] >= st["evaluated"]


def _workloads():
    with open(os.path.join(GOLD, "workloads.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["mixture_d32"])
def test_mixture_config_full(name):
    w = _workloads()[name]
    X = synth.generate(w["kind"], w["n"], w["d"], w["seed"])
    ref = oracle.grid_join(X, w["eps"], 6)
    got, _, _ = _join(X, w["eps"], k=0)
    assert_parity(X, w["eps"], got, ref)


def test_wide_points_plain_and_the_shared_memory_limit():
    """d = 200 joins in the plain form (query tile 64 x 200 doubles); far above
    the shared-memory limit the join reports GJ_ERR_UNSUPPORTED instead of
    launching."""
    X = synth.generate("mixture", 1500, 200, seed=200)
    eps = 1.2
    got, _, _ = _join(X, eps, k=2)
    assert_parity(X, eps, got, oracle.brute(X, eps))
    W = synth.uniform(300, 400, 4)
    with gj.Index(W, 0.5, k=1) as ix:
        st, _ = gj.gj_self_join(ix.h, None)
        assert st == gj.GJ_ERR_UNSUPPORTED
