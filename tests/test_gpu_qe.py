"""The similarity join Q join_eps E (Sec. 3.1) on the GPU against the oracle's
nested loop over Q x E, through the C ABI.

The GPU sums in REORDER order with fused multiply-add, the oracle in the
original order without: the two pair sets may differ only on pairs whose
squared distance lies within 1e-12 relative of fl(eps^2); every such pair is
listed, any other difference fails.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import TIE_REL, keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")


def _assert_qe_parity(Q, E, eps, got):
    ref = oracle.brute_qe(Q, E, eps)
    g, r = keys(got), keys(ref)
    assert g.size == 0 or np.all(np.diff(g.astype(np.int64)) != 0), "duplicate pairs"
    e2 = eps * eps
    bad = []
    for k in np.concatenate([np.setdiff1d(r, g, assume_unique=True), np.setdiff1d(g, r, assume_unique=True)]):
        a, b = int(k >> np.uint64(32)), int(k & np.uint64(0xFFFFFFFF))
        s = oracle.sqdist(Q[a], E[b])
        if abs(s - e2) > TIE_REL * e2:
            bad.append((a, b, s))
    assert not bad, f"pairs outside the tie band differ: {bad[:5]}"
    return r.size


@pytest.mark.parametrize("kind,nq,ne,d,eps,k", [
    ("uniform", 3000, 5000, 8, 0.25, 3),
    ("mixture", 2500, 7000, 32, 0.33, 5),
    ("skewed", 4000, 6000, 18, 0.12, 6),
    ("exponential", 2000, 5000, 16, 0.06, 4),
    ("uniform", 700, 1300, 3, 0.05, 2),
    ("uniform", 1, 4000, 5, 0.3, 0),
])
def test_qe_against_nested_loop(kind, nq, ne, d, eps, k):
    E = synth.generate(kind, ne, d, seed=ne + d)
    Q = synth.generate(kind, nq, d, seed=nq * 3 + d)
    with gj.Index(E, eps, k=k) as ix:
        got = ix.join_qe(Q)
        st = ix.stats()
    m = _assert_qe_parity(Q, E, eps, got)
    assert st["pairs"] == len(got)
    assert len(got) <= st["candidates"] <= nq * ne
    assert len(got) > 0 or m == 0


def test_qe_queries_outside_the_entry_range():
    E = synth.uniform(4000, 6, 3)
    Q = synth.uniform(1500, 6, 4) * 1.6 - 0.3        # overhangs the entries' box on every side
    with gj.Index(E, 0.2, k=4) as ix:
        got = ix.join_qe(Q)
    _assert_qe_parity(Q, E, 0.2, got)


def test_qe_with_q_equal_e_is_the_self_join():
    X = synth.mixture(5000, 16, 8)
    with gj.Index(X, 0.2, k=0) as ix:
        qe = keys(ix.join_qe(X))
        self_join = keys(ix.join())
    assert np.array_equal(qe, self_join)


@pytest.mark.parametrize("flags", [0, gj.GJ_REORDER, gj.GJ_SORTIDU, gj.GJ_SHORTC, gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER])
def test_qe_flags(flags):
    E = synth.skewed(5000, 18, 21)
    Q = synth.skewed(2000, 18, 22)
    with gj.Index(E, 0.1, k=3, flags=flags) as ix:
        got = ix.join_qe(Q)
    _assert_qe_parity(Q, E, 0.1, got)


def test_qe_device_buffers_capacity_and_errors():
    E = synth.uniform(3000, 8, 5)
    Q = synth.uniform(2000, 8, 6)
    Qd = torch.from_numpy(Q).cuda()
    with gj.Index(E, 0.3, k=2) as ix:
        st, m = gj.gj_join_qe(ix.h, Qd, None)
        assert st == gj.GJ_OK and m > 0
        out = torch.full((m + 4, 2), -1, dtype=torch.int32, device="cuda")
        st, m2 = gj.gj_join_qe(ix.h, Qd, out)
        assert st == gj.GJ_OK and m2 == m
        assert int(out[m:].min().item()) == -1
        _assert_qe_parity(Q, E, 0.3, out[:m].cpu().numpy().view(np.uint32))
        small = torch.empty((m - 1, 2), dtype=torch.int32, device="cuda")
        st, m3 = gj.gj_join_qe(ix.h, Qd, small)
        assert st == gj.GJ_ERR_CAPACITY and m3 == m
        bad = Q.copy()
        bad[7, 3] = np.nan
        st, _ = gj.gj_join_qe(ix.h, bad, None)
        assert st == gj.GJ_ERR_NONFINITE
        st, m0 = gj.gj_join_qe(ix.h, np.zeros((0, 8)), None)
        assert st == gj.GJ_OK and m0 == 0


def test_qe_pinned_host_output():
    E = synth.uniform(3000, 8, 5)
    Q = synth.uniform(2000, 8, 6)
    with gj.Index(E, 0.3, k=2) as ix:
        st, m = gj.gj_join_qe(ix.h, Q, None)
        assert st == gj.GJ_OK and m > 0
        host = torch.full((m + 4, 2), -1, dtype=torch.int32).pin_memory()
        st, m2 = gj.gj_join_qe(ix.h, Q, host)
        assert st == gj.GJ_OK and m2 == m
        assert int(host[m:].min()) == -1
        _assert_qe_parity(Q, E, 0.3, host[:m].numpy().view(np.uint32))
        small = torch.empty((m - 1, 2), dtype=torch.int32).pin_memory()
        st, m3 = gj.gj_join_qe(ix.h, Q, small)
        assert st == gj.GJ_ERR_CAPACITY and m3 == m


# ---------------------------------------------------------------------------
# Tensor-core form: an index built with GJ_TC_FILTER runs Q join_eps E through
# the tensor-core filter (query A rows, entry B rows under one centre and one
# scale) and its FP64 recheck.  The recheck is the plain kernel's sum in the
# same order, so the pair set equals the plain form's exactly, and both match
# the nested loop up to the tie band.

TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


def _qe_keys(ix, Q):
    return keys(ix.join_qe(Q))


def _near(E, nq, sd, seed):
    """nq points scattered (normal, sd per coordinate) about random rows of E."""
    rng = np.random.default_rng(seed)
    return E[rng.integers(0, len(E), nq)] + rng.standard_normal((nq, E.shape[1])) * sd


# sd > 0: half the queries scattered about entries (a clustered set drawn with
# another seed has other clusters); pair counts 38 - 32,597
@pytest.mark.parametrize("kind,nq,ne,d,eps,sd", [
    ("uniform", 3000, 5000, 8, 0.25, 0),
    ("mixture", 2500, 7000, 32, 0.33, 0.05),
    ("skewed", 4000, 6000, 18, 0.12, 0.02),
    ("exponential", 2000, 5000, 16, 0.06, 0),
    ("uniform", 700, 1300, 64, 2.6, 0),
    ("mixture", 1500, 2500, 124, 0.6, 0.04),
    ("uniform", 1, 4000, 5, 0.3, 0),
    ("uniform", 129, 257, 12, 0.7, 0),          # ragged: a few partial A and B tiles
])
def test_qe_tc_equals_plain_and_the_nested_loop(kind, nq, ne, d, eps, sd):
    E = synth.generate(kind, ne, d, seed=ne + d)
    Q = synth.generate(kind, nq, d, seed=nq * 3 + d)
    if sd:
        Q[: nq // 2] = _near(E, nq // 2, sd, nq + d)
    with gj.Index(E, eps, k=0) as ip:
        ref = _qe_keys(ip, Q)
    with gj.Index(E, eps, k=0, flags=TC) as it:
        got = it.join_qe(Q)
        st = it.stats()
    assert np.array_equal(keys(got), ref)
    _assert_qe_parity(Q, E, eps, got)
    assert st["pairs"] == len(got)
    assert st["tc_survivors"] >= len(got)          # every pair passed the filter
    assert st["evaluated"] >= len(got)


@pytest.mark.parametrize("scale", [1.0, 1.6, 40.0])
def test_qe_tc_queries_beyond_the_entries(scale):
    # scale 1.6 overhangs the entries' box on every side (a larger radius
    # about the centre: the queries' scale may differ from the entries'); at
    # 40 the scale is several powers of two smaller and the entry rows are
    # re-packed, with a looser filter but the same exact result
    E = synth.uniform(5000, 16, 3)
    Q = (synth.uniform(1500, 16, 4) - 0.5) * scale + 0.5
    Q[:200] = E[:200] + 0.01                      # some queries with neighbours in every case
    eps = 0.45
    with gj.Index(E, eps, k=0) as ip:
        ref = _qe_keys(ip, Q)
    with gj.Index(E, eps, k=0, flags=TC) as it:
        got = it.join_qe(Q)
    assert np.array_equal(keys(got), ref)
    _assert_qe_parity(Q, E, eps, got)
    assert len(got) >= 200


def test_qe_tc_planted_pairs_at_the_radius():
    # pairs at eps (1 - 2^-40) from entries farthest from the centre: the
    # tightest case of the filter's margin
    rng = np.random.default_rng(5)
    d, eps = 48, 0.3
    E = synth.uniform(6000, d, 11)
    c = 0.5 * (E.min(0) + E.max(0))
    far = np.argsort(-np.linalg.norm(E - c, axis=1))[:300]
    u = rng.standard_normal((300, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Q = E[far] + u * (eps * (1 - 2.0 ** -40))
    with gj.Index(E, eps, k=0, flags=TC) as it:
        pairs = it.join_qe(Q)
    _assert_qe_parity(Q, E, eps, pairs)
    want = (np.arange(300, dtype=np.uint64) << np.uint64(32)) | far.astype(np.uint64)
    assert np.isin(want, keys(pairs)).all()


def test_qe_tc_capacity_host_output_and_empty():
    E = synth.mixture(6000, 24, 8)
    Q = _near(E, 3000, 0.03, 9)
    eps = 0.2
    Qd = torch.from_numpy(Q).cuda()
    with gj.Index(E, eps, k=0, flags=TC) as it:
        st, m = gj.gj_join_qe(it.h, Qd, None)
        assert st == gj.GJ_OK and m > 0
        out = torch.full((m + 4, 2), -1, dtype=torch.int32, device="cuda")
        st, m2 = gj.gj_join_qe(it.h, Qd, out)
        assert st == gj.GJ_OK and m2 == m
        assert int(out[m:].min().item()) == -1
        got = out[:m].cpu().numpy().view(np.uint32)
        _assert_qe_parity(Q, E, eps, got)
        small = torch.empty((m // 2, 2), dtype=torch.int32, device="cuda")
        st, m3 = gj.gj_join_qe(it.h, Qd, small)
        assert st == gj.GJ_ERR_CAPACITY and m3 == m
        # the pairs written before the capacity ran out are pairs of the result
        part = keys(small.cpu().numpy().view(np.uint32))
        assert np.isin(part, keys(got)).all()
        host = np.full((m + 4, 2), 0xFFFFFFFF, dtype=np.uint32)
        st, m4 = gj.gj_join_qe(it.h, Q, host)
        assert st == gj.GJ_OK and m4 == m
        assert np.array_equal(keys(host[:m]), keys(got)) and (host[m:] == 0xFFFFFFFF).all()
        st, m0 = gj.gj_join_qe(it.h, np.zeros((0, 24)), None)
        assert st == gj.GJ_OK and m0 == 0
        far = np.full((10, 24), 1e6)                 # no entry anywhere near
        st, mf = gj.gj_join_qe(it.h, far, None)
        assert st == gj.GJ_OK and mf == 0


def test_qe_tc_with_q_equal_e_is_the_self_join():
    X = synth.mixture(5000, 16, 8)
    with gj.Index(X, 0.2, k=0, flags=TC) as it:
        assert np.array_equal(_qe_keys(it, X), keys(it.join()))


def test_qe_tc_paper_scale_sampled_queries():
    # the bench's workload: 200,000 uniform queries against the 2M-point d = 16
    # set at its eps; every pair of the first 300 queries against the nested
    # loop, the whole set against the plain form's count
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")) as f:
        w = json.load(f)["paper_d16"]
    E = synth.uniform(2_000_000, 16, w["seed"])
    Q = synth.uniform(200_000, 16, w["seed"] + 7919)
    Ed, Qd = torch.from_numpy(E).cuda(), torch.from_numpy(Q).cuda()
    with gj.Index(Ed, w["eps"], k=0) as ip:
        st, mp = gj.gj_join_qe(ip.h, Qd, None)
        assert st == gj.GJ_OK
    with gj.Index(Ed, w["eps"], k=0, flags=TC) as it:
        out = torch.empty((mp + 16, 2), dtype=torch.int32, device="cuda")
        st, m = gj.gj_join_qe(it.h, Qd, out)
        assert st == gj.GJ_OK and m == mp
        got = out[:m].cpu().numpy().view(np.uint32)
    sel = got[got[:, 0] < 300]
    _assert_qe_parity(Q[:300], E, w["eps"], sel)
