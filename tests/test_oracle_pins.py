"""Pins of the CPU oracle against what the paper and mathematics fix.

Every expected value here comes from the paper (worked examples, printed
constants; fixtures under tests/golden/ carry their citation) or from an
argument independent of the oracle's code: closed-form counts on integer
lattices, exact integer arithmetic, a sorted two-pointer sweep in one
dimension.  None comes from the CUDA library.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Fig. 1 (Sec. 3.2.1): linearised ids and the adjacent-cell search
# ---------------------------------------------------------------------------

def _fig1_points(g):
    xy = np.array(g["dots_tikz_xy"], dtype=np.float64)
    return np.stack([7.0 - xy[:, 1], xy[:, 0]], axis=1)   # (row_coord, col_coord)


def test_fig1_linear_ids_of_shaded_cells():
    g = _gold("fig1_grid.json")
    for x, y, cid in g["shaded_tikz_x_y_id"]:
        row, col = 6 - y, x
        assert oracle.linearise([row, col], g["ncells"]) == cid


def test_fig1_points_fill_exactly_the_shaded_cells():
    g = _gold("fig1_grid.json")
    P = _fig1_points(g)
    c = oracle.cell_coords(P, 2, g["origin"], g["eps"])
    ids = {oracle.linearise(ci, g["ncells"]) for ci in c}
    assert ids == {s[2] for s in g["shaded_tikz_x_y_id"]}


def test_fig1_query_in_cell_24_searches_18_23_24_32():
    g = _gold("fig1_grid.json")
    ids = sorted(s[2] for s in g["shaded_tikz_x_y_id"])
    q = g["query_cell"]
    coord = [q // 7, q % 7]
    got = oracle.adjacent_nonempty(ids, coord, g["ncells"])
    assert list(got) == g["adjacent_nonempty_of_query_cell"]


def test_fig1_join_equals_nested_loop():
    g = _gold("fig1_grid.json")
    P = _fig1_points(g)
    ref = oracle.brute(P, g["eps"])
    for k in (0, 1, 2):
        assert np.array_equal(oracle.grid_join(P, g["eps"], k), ref)


# ---------------------------------------------------------------------------
# Fig. 2 (Sec. 4.2): REORDER
# ---------------------------------------------------------------------------

def test_fig2_reorder_partial_pin():
    g = _gold("fig2_reorder.json")
    F = np.array(g["columns"], dtype=np.float64).T / g["scale"]
    perm = [int(p) + 1 for p in oracle.reorder_perm(F)]        # 1-based like the figure
    assert set(perm[:3]) == set(g["pinned_top3_set"])
    assert perm[3:] == g["pinned_bottom_order"]
    c = oracle.cell_coords(F, 6, np.zeros(6), g["eps"])
    assert [len(set(c[:, j])) for j in range(6)] == g["pinned_cells_per_dim"]
    # after REORDER the first three dimensions each span 5 cells (text after Fig. 2)
    Fr = F[:, np.array(perm) - 1]
    cr = oracle.cell_coords(Fr, 3, np.zeros(3), g["eps"])
    assert [len(set(cr[:, j])) for j in range(3)] == [5, 5, 5]


def test_reorder_ties_keep_lower_index():
    X = np.zeros((4, 5))
    X[:, 1] = [0, 1, 0, 1]
    X[:, 3] = [1, 0, 1, 0]      # same variance as dim 1
    X[:, 4] = [0, 2, 0, 2]      # largest
    assert list(oracle.reorder_perm(X)) == [4, 1, 3, 0, 2]


def test_population_variance_closed_form():
    # 0..m-1 has population variance (m^2-1)/12
    m = 101
    X = np.arange(m, dtype=np.float64)[:, None]
    _, v = oracle.variance(X)
    assert v[0] == pytest.approx((m * m - 1) / 12.0, rel=1e-15)


# ---------------------------------------------------------------------------
# Printed constants
# ---------------------------------------------------------------------------

def test_index_loss_5_3_is_88_9_percent():
    c = _gold("paper_constants.json")["index_loss"]
    assert round(100.0 * oracle.index_loss(c["n"], c["k"]), c["printed_digits"]) == c["value_percent"]
    assert oracle.index_loss(4, 4) == 0.0


def test_selectivity_excludes_self_pairs():
    X = np.arange(10, dtype=np.float64)[:, None] * 10.0    # no two points within 1
    R = oracle.brute_count(X, 1.0)
    assert R == 10 and oracle.selectivity(R, 10) == 0.0


# ---------------------------------------------------------------------------
# Closed forms on integer lattices (exact in every summation order)
# ---------------------------------------------------------------------------

def lattice_pairs_closed_form(L: int, d: int, E: int) -> int:
    """Ordered pairs (p,q) of {0..L-1}^d with |p-q|^2 <= E: sum over integer
    offsets o of prod_j (L - |o_j|), by convolution over the squared norm."""
    per_dim = {}
    for o in range(-(L - 1), L):
        t = o * o
        if t <= E:
            per_dim[t] = per_dim.get(t, 0) + (L - abs(o))
    poly = {0: 1}
    for _ in range(d):
        nxt = {}
        for a, ca in poly.items():
            for b, cb in per_dim.items():
                if a + b <= E:
                    nxt[a + b] = nxt.get(a + b, 0) + ca * cb
        poly = nxt
    return sum(poly.values())


def full_lattice(L, d):
    g = np.stack(np.meshgrid(*[np.arange(L)] * d, indexing="ij"), axis=-1)
    return g.reshape(-1, d).astype(np.float64)


def test_closed_form_helper_matches_simple_formula():
    for L, d in ((3, 2), (5, 4), (4, 6)):
        assert lattice_pairs_closed_form(L, d, 1) == L ** d + 2 * d * (L - 1) * L ** (d - 1)


@pytest.mark.parametrize("L,d", [(5, 3), (4, 5), (3, 8)])
@pytest.mark.parametrize("eps,E", [(1.0, 1), (2.0, 4), (3.0, 9)])
def test_full_lattice_counts(L, d, eps, E):
    X = full_lattice(L, d)
    want = lattice_pairs_closed_form(L, d, E)
    assert oracle.brute_count(X, eps) == want
    for k in (0, 1, min(d, 3), min(d, 6)):
        assert oracle.grid_count(X, eps, k)["R"] == want


def test_boundary_is_inclusive_and_uses_rounded_eps_squared():
    L, d = 4, 4
    X = full_lattice(L, d)
    # fl(sqrt2)^2 rounds to 2 + 2^-51 >= 2: distance-sqrt2 pairs are in R
    e = math.sqrt(2.0)
    assert e * e > 2.0
    assert oracle.brute_count(X, e) == lattice_pairs_closed_form(L, d, 2)
    # just below 1: only the self-pairs
    below = np.nextafter(1.0, 0.0)
    assert oracle.brute_count(X, below) == L ** d
    assert oracle.grid_count(X, below, 3)["R"] == L ** d


def test_random_lattice_subset_exact_integer_reference():
    # on small integers every difference, square and partial sum is exact, so
    # R is {(i,j): integer |x_i - x_j|^2 <= fl(eps^2)} whatever the order
    X = synth.lattice(700, 5, seed=7, side=6)
    Xi = X.astype(np.int64)
    dif = Xi[:, None, :] - Xi[None, :, :]
    sq = (dif * dif).sum(-1)
    for eps in (1.0, 2.0 ** 0.5, 3.0 ** 0.5, 2.0, 5.0 ** 0.5):
        want = np.argwhere(sq <= eps * eps).astype(np.uint32)
        got = oracle.grid_join(X, eps, 3)
        assert np.array_equal(got, want)


def test_d1_two_pointer_sweep():
    # dyadic data and eps: every difference and square is exact
    z = synth.splitmix64(11, 3000)
    x = ((z >> np.uint64(54)).astype(np.float64)) * 2.0 ** -10        # multiples of 2^-10 in [0,1)
    eps = 3 * 2.0 ** -10
    order = np.argsort(x, kind="stable")
    xs = x[order]
    want = []
    lo = 0
    for a in range(len(xs)):                      # window [xs[a]-eps, xs[a]+eps] by two pointers
        while xs[lo] < xs[a] - eps:
            lo += 1
        hi = a
        while hi + 1 < len(xs) and xs[hi + 1] <= xs[a] + eps:
            hi += 1
        for b in range(lo, hi + 1):
            want.append((order[a], order[b]))
    want = np.array(sorted(want), dtype=np.uint32)
    assert np.array_equal(oracle.brute(x[:, None], eps), want)
    assert np.array_equal(oracle.grid_join(x[:, None], eps, 1), want)


def test_all_duplicates_and_separated_clusters():
    X = np.full((300, 7), 0.25)
    assert oracle.grid_count(X, 1e-3, 4)["R"] == 300 * 300
    a = np.zeros((120, 3))
    b = np.full((80, 3), 5.0)
    a[:, 0] = np.linspace(0, 0.5, 120)            # diameter 0.5 <= eps
    X = np.vstack([a, b])
    assert oracle.grid_count(X, 0.5, 2)["R"] == 120 * 120 + 80 * 80


def test_depth_stats_hand_example():
    # q = 0 against j = 1 (far in dim 0) and j = 2 (far only in the last dim)
    X = np.array([[0.0, 0.0, 0.0, 0.0],
                  [2.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 2.0]])
    ds, pc = oracle.depth_stats(X, 1.0, [0, 1, 2, 3], [0])
    assert (ds, pc) == (1 + 4, 2)
    ds, pc = oracle.depth_stats(X, 1.0, [3, 2, 1, 0], [0])
    assert (ds, pc) == (4 + 1, 2)


# ---------------------------------------------------------------------------
# constructNeighborTable (Alg. 1; Sec. 3.2.2) on the full integer lattice:
# each row is known independently -- the lattice points x + o with integer
# offsets |o|^2 <= E that stay inside the box, ids row-major
# ---------------------------------------------------------------------------

def lattice_row(x, L, E):
    d = len(x)
    r = int(math.isqrt(E))
    offs = np.stack(np.meshgrid(*[np.arange(-r, r + 1)] * d, indexing="ij"), axis=-1).reshape(-1, d)
    offs = offs[(offs * offs).sum(axis=1) <= E]
    y = np.asarray(x) + offs
    y = y[np.all((y >= 0) & (y < L), axis=1)]
    ids = np.zeros(len(y), dtype=np.int64)
    for j in range(d):
        ids = ids * L + y[:, j]
    return np.sort(ids)


@pytest.mark.parametrize("L,d,E", [(4, 3, 2), (5, 2, 4), (3, 4, 1)])
def test_neighbor_table_rows_on_the_lattice(L, d, E):
    X = full_lattice(L, d)
    n = len(X)
    row_start, nbr = oracle.neighbor_table(oracle.brute(X, math.sqrt(E)), n)
    assert row_start[0] == 0 and row_start[-1] == lattice_pairs_closed_form(L, d, E)
    assert np.all(np.diff(row_start) >= 1)            # every point is its own neighbour
    for a in range(n):
        got = nbr[row_start[a]:row_start[a + 1]].astype(np.int64)
        assert np.array_equal(got, lattice_row(X[a].astype(np.int64), L, E)), a


def test_neighbor_table_empty_and_isolated_rows():
    row_start, nbr = oracle.neighbor_table(np.zeros((0, 2), dtype=np.uint32), 3)
    assert list(row_start) == [0, 0, 0, 0] and nbr.size == 0
    X = np.array([[0.0], [10.0], [0.5], [20.0]])
    row_start, nbr = oracle.neighbor_table(oracle.brute(X, 1.0), 4)
    assert list(row_start) == [0, 2, 3, 5, 6]
    assert list(nbr) == [0, 2, 1, 0, 2, 3]


# ---------------------------------------------------------------------------
# Q join_eps E (Sec. 3.1): the self-join is the case Q = E; on integer
# coordinates every term is exact, so an integer reference decides each pair
# ---------------------------------------------------------------------------

def test_qe_with_q_equal_e_is_the_self_join():
    X = synth.mixture(900, 7, 5)
    assert np.array_equal(oracle.brute_qe(X, X, 0.2), oracle.brute(X, 0.2))


@pytest.mark.parametrize("nq,ne,d,side,E2", [(150, 220, 4, 5, 2), (90, 400, 6, 4, 3), (1, 300, 3, 7, 5)])
def test_qe_integer_reference(nq, ne, d, side, E2):
    Q = synth.lattice(nq, d, seed=nq, side=side)
    E = synth.lattice(ne, d, seed=ne + 1, side=side)
    Qi, Ei = Q.astype(np.int64), E.astype(np.int64)
    dif = Qi[:, None, :] - Ei[None, :, :]
    want = np.argwhere((dif * dif).sum(-1) <= E2).astype(np.uint32)
    got = oracle.brute_qe(Q, E, math.sqrt(E2) * (1 + 1e-12))
    assert np.array_equal(got, want)


def test_qe_boundary_is_inclusive():
    Q = synth.lattice(120, 3, seed=31, side=5)
    E = synth.lattice(160, 3, seed=32, side=5)
    dif = Q.astype(np.int64)[:, None, :] - E.astype(np.int64)[None, :, :]
    for eps, E2 in ((1.0, 1), (2.0, 4), (3.0, 9)):
        want = np.argwhere((dif * dif).sum(-1) <= E2).astype(np.uint32)
        assert np.array_equal(oracle.brute_qe(Q, E, eps), want)


def test_qe_orientation_and_far_sets():
    Q = np.array([[0.0], [5.0]])
    E = np.array([[0.5], [10.0], [4.0]])
    assert oracle.brute_qe(Q, E, 1.0).tolist() == [[0, 0], [1, 2]]
    assert oracle.brute_qe(Q + 100.0, E, 1.0).size == 0
    assert oracle.brute_qe(np.zeros((0, 1)), E, 1.0).size == 0


# ---------------------------------------------------------------------------
# One point's neighbours by the definition (Sec. 3.1): the checker the
# full-size tests use per sampled query.  On the full integer lattice each row
# is known independently (lattice_row); on a random lattice subset exact
# integer arithmetic decides every pair; at eps = 2 and 3 the boundary is
# exact, so a strict comparison or an unsquared eps changes the row.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,d", [(4, 3), (5, 2), (3, 4)])
@pytest.mark.parametrize("eps,E", [(1.0, 1), (math.sqrt(2.0), 2), (2.0, 4), (3.0, 9)])
def test_query_neighbors_rows_on_the_lattice(L, d, eps, E):
    X = full_lattice(L, d)
    for q in range(len(X)):
        got = oracle.query_neighbors(X, eps, q).astype(np.int64)
        assert np.array_equal(got, lattice_row(X[q].astype(np.int64), L, E)), q


def test_query_neighbors_exact_integer_reference():
    X = synth.lattice(500, 6, seed=13, side=5)
    Xi = X.astype(np.int64)
    for q in (0, 1, 77, 250, 499):
        dif = Xi - Xi[q]
        sq = (dif * dif).sum(-1)
        for eps, E2 in ((1.0, 1), (2.0, 4), (math.sqrt(5.0) * (1 + 1e-12), 5)):
            want = np.flatnonzero(sq <= E2)
            assert np.array_equal(oracle.query_neighbors(X, eps, q).astype(np.int64), want)


@pytest.mark.parametrize("kind", ["uniform", "mixture", "skewed"])
def test_query_neighbors_equal_the_rows_of_the_nested_loop(kind):
    X = synth.generate(kind, 1500, 9, 21)
    eps = {"uniform": 0.45, "mixture": 0.12, "skewed": 0.15}[kind]
    pairs = oracle.brute(X, eps)
    for q in (0, 3, 700, 1499):
        want = pairs[pairs[:, 0] == q, 1]
        assert np.array_equal(oracle.query_neighbors(X, eps, q), want), q
