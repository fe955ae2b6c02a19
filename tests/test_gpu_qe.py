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
