"""Invariants of the self-join result, checked on the CPU oracle.

The paper's filters (grid over k dims, REORDER, SORTIDU, SHORTC) only skip
work, so the result must not depend on them (Sec. 4.1–4.4); the result is
symmetric and holds every self-pair (Sec. 5.2); it grows with ε; scaling
points and ε by a power of two changes no rounding, hence no pair.
"""
import numpy as np
import pytest

import oracle
import synth


def _as_set(p):
    return set(map(tuple, p.tolist()))


CASES = [
    ("uniform", 1500, 16, 0.9),
    ("uniform", 1200, 5, 0.25),
    ("mixture", 1500, 32, 0.35),
    ("skewed", 2000, 18, 0.15),
    ("exponential", 1500, 16, 0.05),
]


@pytest.mark.parametrize("kind,n,d,eps", CASES)
def test_grid_method_equals_nested_loop(kind, n, d, eps):
    X = synth.generate(kind, n, d, seed=n + d)
    ref = oracle.brute(X, eps)
    assert len(ref) > n           # some non-self pairs
    for k in sorted({min(k, d) for k in (0, 1, 2, 4, 6)}):
        for flags in (0, oracle.REORDER, oracle.SORTIDU, oracle.SHORTC, oracle.ALL):
            got = oracle.grid_join(X, eps, k, flags)
            assert np.array_equal(got, ref), (k, flags)


@pytest.mark.parametrize("kind,n,d,eps", CASES[:3])
def test_symmetry_and_self_pairs(kind, n, d, eps):
    X = synth.generate(kind, n, d, seed=3)
    p = oracle.grid_join(X, eps, 4)
    s = _as_set(p)
    assert all((b, a) in s for a, b in s)
    assert all((i, i) in s for i in range(n))


def test_monotone_in_eps():
    X = synth.uniform(1500, 8, 5)
    prev = set()
    for eps in (0.1, 0.2, 0.3, 0.45, 0.6):
        cur = _as_set(oracle.grid_join(X, eps, 4))
        assert prev <= cur
        prev = cur


@pytest.mark.parametrize("s", [-7, 3, 20])
def test_power_of_two_scaling(s):
    X = synth.mixture(1500, 16, 9)
    ref = oracle.brute(X, 0.3)
    f = 2.0 ** s
    assert np.array_equal(oracle.grid_join(X * f, 0.3 * f, 5), ref)


def test_column_permutation_on_exact_data():
    X = synth.lattice(900, 6, seed=2, side=5)
    ref = oracle.brute(X, 2.0)
    rng_perm = np.argsort(synth.uniform01(4, 6))
    assert np.array_equal(oracle.brute(X[:, rng_perm], 2.0), ref)
    assert np.array_equal(oracle.grid_join(X[:, rng_perm], 2.0, 3), ref)


def test_k_equals_d_and_tiny_inputs():
    X = synth.uniform(400, 3, 8)
    ref = oracle.brute(X, 0.2)
    assert np.array_equal(oracle.grid_join(X, 0.2, 3), ref)
    assert len(oracle.brute(np.zeros((0, 3)), 0.1)) == 0
    one = oracle.brute(np.zeros((1, 3)), 0.1)
    assert one.tolist() == [[0, 0]]


def test_candidate_count_single_cell_is_all_pairs():
    X = synth.uniform(800, 4, 1)
    st = oracle.grid_count(X, 2.0, 3)     # eps > range: one cell per dimension
    assert st["nonempty_cells"] == 1
    assert st["candidates"] == 800 * 799 // 2
