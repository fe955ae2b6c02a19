"""The device neighbour table (constructNeighborTable of Alg. 1, Sec. 3.2.2)
against the oracle's table of the same pair set.

Rows are in original point order and sorted, so where the GPU and oracle pair
sets agree (everything outside the tie band) the two tables are equal element
by element; where a tie pair differs, the rows are compared after removing it.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


def _check(X, eps, flags, k=0):
    n = len(X)
    ref = oracle.brute(X, eps)
    with gj.Index(X, eps, k=k, flags=flags) as ix:
        rs_d, nbr_d = ix.neighbor_table()
        rs, nbr = rs_d.cpu().numpy(), nbr_d.cpu().numpy().view(np.uint32)
        pairs = ix.join()
    res = compare(X, eps, pairs, ref)
    assert not res["bad"]
    if not res["ties"]:
        ref_rs, ref_nbr = oracle.neighbor_table(ref, n)
        assert np.array_equal(rs, ref_rs)
        assert np.array_equal(nbr, ref_nbr)
    else:
        # the table must be the table of the GPU's own pair set
        own_rs, own_nbr = oracle.neighbor_table(pairs, n)
        assert np.array_equal(rs, own_rs) and np.array_equal(nbr, own_nbr)
    return rs, nbr


def test_tiny_config_table():
    w = json.load(open(os.path.join(GOLD, "workloads.json")))["tiny"]
    X = synth.uniform(w["n"], w["d"], w["seed"])
    rs, nbr = _check(X, w["eps"], gj.GJ_DEFAULT_FLAGS, k=6)
    assert rs[-1] == w["R"]


@pytest.mark.parametrize("kind,n,d,eps,flags", [
    ("mixture", 6000, 32, 0.33, TC),
    ("skewed", 9000, 18, 0.1, gj.GJ_DEFAULT_FLAGS),
    ("uniform", 70000, 3, 0.01, gj.GJ_DEFAULT_FLAGS),       # n > 2^16: keys wider than 32 bits
    ("uniform", 1, 4, 0.5, gj.GJ_DEFAULT_FLAGS),
])
def test_shapes(kind, n, d, eps, flags):
    X = synth.generate(kind, n, d, seed=n + d)
    rs, nbr = _check(X, eps, flags)
    assert rs[0] == 0 and np.all(np.diff(rs) >= 1)


def test_capacity_and_host_buffers_rejected():
    X = synth.uniform(3000, 8, 4)
    with gj.Index(X, 0.3) as ix:
        m = ix.count()
        rs = torch.empty(3001, dtype=torch.int64, device="cuda")
        small = torch.empty(m - 1, dtype=torch.int32, device="cuda")
        st, c = gj.gj_neighbor_table(ix.h, rs, small)
        assert st == gj.GJ_ERR_CAPACITY and c == m
        st, _ = gj.gj_neighbor_table(ix.h, torch.empty(3001, dtype=torch.int64), small)
        assert st == gj.GJ_ERR_INVALID_ARG
