"""The autotuner: its picks are valid settings, and every setting it may pick
gives the oracle's pair set.

The tuner only chooses among settings that filter work (k, query block,
candidate tile, form, b_s); none of them may change R.  So each test checks
the pick's range and then the result of the tuned index against the oracle.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import assert_parity, keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")
torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


@pytest.mark.parametrize("qb,tile", [(8, 32), (33, 64), (64, 32), (64, 64), (120, 32), (128, 64)])
def test_plain_tiles_against_oracle(qb, tile):
    X = synth.generate("mixture", 5000, 32, seed=qb * 131 + tile)
    eps = 0.33
    ref = oracle.grid_join(X, eps, 4)
    with gj.Index(X, eps, k=4, query_block=qb, tile=tile) as ix:
        got = ix.join()
        assert ix.info()["work_items"] >= -(-5000 // qb)
    assert_parity(X, eps, got, ref)


@pytest.mark.parametrize("qb", [0, 16, 64, 120])
def test_tc_query_blocks_equal_plain(qb):
    X = synth.generate("uniform", 9000, 16, seed=qb)
    eps = 0.45
    with gj.Index(X, eps, k=2) as ip:
        plain = keys(ip.join())
    with gj.Index(X, eps, k=2, flags=TC, query_block=qb) as it:
        tc = keys(it.join())
    assert np.array_equal(plain, tc)


def test_autotune_tiny_pick_and_result():
    w = json.load(open(os.path.join(GOLD, "workloads.json")))["tiny"]
    X = synth.uniform(w["n"], w["d"], w["seed"])
    r = gj.gj_autotune(X, w["eps"])
    assert 1 <= r["k"] <= 8 and r["trials"] >= 3
    assert r["query_block"] in (0, 64) and r["tile"] in (32, 64)
    assert r["flags"] & gj.GJ_TC_FILTER == 0
    assert r["join_ms"] > 0 and r["build_ms"] > 0
    # the trial's extrapolated |R| is an estimate; the exact count is pinned
    assert 0.3 * w["R"] < r["est_pairs"] < 3.0 * w["R"]
    with gj.Index(X, w["eps"], k=r["k"], query_block=r["query_block"], tile=r["tile"],
                  batch_pairs=r["batch_pairs"]) as ix:
        got = ix.join()
    assert_parity(X, w["eps"], got, oracle.brute(X, w["eps"]))


def test_build_with_autotune_flag_returns_the_pick():
    X = synth.generate("skewed", 30000, 18, seed=5)
    eps = 0.05
    ref = oracle.grid_join(X, eps, 6)
    with gj.Index(X, eps, k=0, flags=gj.GJ_DEFAULT_FLAGS | gj.GJ_AUTOTUNE) as ix:
        info = ix.info()
        assert 1 <= info["k"] <= 8
        got = ix.join()                          # host output: the tuned b_s applies
        st = ix.stats()
    assert st["batch_pairs"] > 0
    assert_parity(X, eps, got, ref)


def test_autotune_both_forms():
    X = synth.generate("mixture", 20000, 32, seed=3)
    eps = 0.3
    r = gj.gj_autotune(X, eps, _cfg(gj.GJ_DEFAULT_FLAGS | gj.GJ_TUNE_FORM))
    assert r["trials"] >= 5
    tc = bool(r["flags"] & gj.GJ_TC_FILTER)
    assert (not tc) or 1 <= r["k"] <= 3
    flags = gj.GJ_DEFAULT_FLAGS | (gj.GJ_TC_FILTER if tc else 0)
    with gj.Index(X, eps, k=r["k"], flags=flags, query_block=r["query_block"], tile=r["tile"]) as ix:
        got = ix.join()
    assert_parity(X, eps, got, oracle.grid_join(X, eps, 5))


def test_autotune_device_input_and_empty():
    X = torch.from_numpy(synth.uniform(4000, 8, 2)).cuda()
    r = gj.gj_autotune(X, 0.2)
    assert 1 <= r["k"] <= 8
    r0 = gj.gj_autotune(np.zeros((0, 4)), 0.5)
    assert r0["est_pairs"] == 0 and r0["batch_pairs"] == 0


def _cfg(flags):
    c = gj.gj_config_init()
    c.flags = flags
    return c


def test_batch_autotune_picks_and_cache():
    jobs = []
    for j, js in enumerate(synth.many_jobs(count=10, seed=21, n_lo=500, n_hi=20000)):
        X = synth.generate(js.kind, js.n, js.d, js.seed)
        jobs.append((X, 0.08 if js.kind != "uniform" else 0.35, 0))
    cfg = _cfg(gj.GJ_DEFAULT_FLAGS | gj.GJ_AUTOTUNE)
    b = gj.gj_batch_build(jobs, cfg)
    try:
        ks = gj.gj_batch_get_k(b, len(jobs))
        assert all(1 <= k <= 3 for k in ks)
        st, counts = gj.gj_batch_self_join(b, len(jobs))
        assert st == gj.GJ_OK
        outs = [torch.empty((c + 1, 2), dtype=torch.int32, device="cuda") for c in counts]
        st, _ = gj.gj_batch_self_join(b, len(jobs), outs)
        assert st == gj.GJ_OK
        for j in range(len(jobs)):
            X, eps, _ = jobs[j]
            got = outs[j][:counts[j]].cpu().numpy().view(np.uint32)
            assert_parity(X, eps, got, oracle.brute(X, eps))
    finally:
        gj.gj_batch_free(b)
    # the same shapes again: the remembered picks, no trials
    before = gj.gj_kernel_launches()
    b2 = gj.gj_batch_build(jobs, cfg)
    try:
        assert gj.gj_batch_get_k(b2, len(jobs)) == ks
        build_launches = gj.gj_kernel_launches() - before
    finally:
        gj.gj_batch_free(b2)
    before = gj.gj_kernel_launches()
    b3 = gj.gj_batch_build([(X, e, k) for (X, e, _), k in zip(jobs, ks)])
    gj.gj_batch_free(b3)
    assert build_launches == gj.gj_kernel_launches() - before
