"""Plant plausible mistakes in a copy of the oracle and check the pins catch them.

Each mutant is the oracle's C source with one edit (a dropped term, a strict
inequality, a wrong offset, a reversed order ...), compiled to a temporary
library; the pins below must reject every mutant while the real oracle passes
them.  This runs on the CPU only.
"""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import full_lattice, lattice_pairs_closed_form, lattice_row

SRC = os.path.join(os.path.dirname(oracle.__file__), "gj_oracle.c")

MUTANTS = {
    "drop_last_dim": ("    for (int j = 0; j < d; ++j) {\n        double t = a[j] - b[j];\n        s = s + t * t;\n    }\n    return s;\n}\n\n/* Same sum",
                      "    for (int j = 0; j < d - 1; ++j) {\n        double t = a[j] - b[j];\n        s = s + t * t;\n    }\n    return s;\n}\n\n/* Same sum"),
    "strict_brute": ("a->X + j * a->d, a->d) <= a->e2)", "a->X + j * a->d, a->d) < a->e2)"),
    "strict_grid": ("if (sd <= a->e2) {", "if (sd < a->e2) {"),
    "offsets_0_to_2": ("nb[j] = ci[j] + (r % 3) - 1;", "nb[j] = ci[j] + (r % 3);"),
    "reorder_ascending": ("while (b >= 0 && var[perm[b]] < var[p]) {", "while (b >= 0 && var[perm[b]] > var[p]) {"),
    "linearise_col_major": ("        id = id * ncells[j] + c[j];", "        id = id + c[j] * (j ? ncells[j - 1] : 1);"),
    "sortidu_one_sided": ("while (stop < e && a->Y[(size_t)a->order[stop] * d + a->u] - ui <= a->ew)",
                          "while (stop < e && a->Y[(size_t)a->order[stop] * d + a->u] - ui <= 0.0)"),
    "eps_not_squared": ("    double e2 = eps * eps;\n    brute_arg", "    double e2 = eps;\n    brute_arg"),
    "shortc_wrong_sign": ("        if (s > e2)\n            return s;", "        if (s < e2)\n            return s;"),
    "query_strict": ("if (gjo_sqdist(X + q * d, X + j * d, d) <= e2) {",
                     "if (gjo_sqdist(X + q * d, X + j * d, d) < e2) {"),
    "query_eps_not_squared": ("    double e2 = eps * eps;\n    int64_t c = 0;", "    double e2 = eps;\n    int64_t c = 0;"),
    "query_row_offset": ("if (gjo_sqdist(X + q * d, X + j * d, d) <= e2) {",
                         "if (gjo_sqdist(X + q, X + j * d, d) <= e2) {"),
    "qe_strict": ("a->E + j * a->d, a->d) <= a->e2)", "a->E + j * a->d, a->d) < a->e2)"),
    "qe_swapped_orientation": ("kv_push(&a->out, ((uint64_t)i << 32) | (uint64_t)j);\n    return NULL;\n}\n\n/* Every pair",
                               "kv_push(&a->out, ((uint64_t)j << 32) | (uint64_t)i);\n    return NULL;\n}\n\n/* Every pair"),
}


def _pins_pass() -> bool:
    """A compact subset of the pins; True iff all hold."""
    try:
        L, d = 4, 4
        X = full_lattice(L, d)
        if oracle.brute_count(X, 1.0) != lattice_pairs_closed_form(L, d, 1):
            return False
        if oracle.brute_count(X, math.sqrt(2.0)) != lattice_pairs_closed_form(L, d, 2):
            return False
        if oracle.grid_count(X, 2.0, 3)["R"] != lattice_pairs_closed_form(L, d, 4):
            return False
        # Fig. 1
        if oracle.linearise([3, 3], [7, 7]) != 24 or oracle.linearise([2, 4], [7, 7]) != 18:
            return False
        ids = sorted([14, 36, 23, 8, 47, 24, 18, 32, 34, 2])
        if list(oracle.adjacent_nonempty(ids, [3, 3], [7, 7])) != [18, 23, 24, 32]:
            return False
        # Fig. 2 top-3 set
        cols = np.array([[1.2, 1.25, 1.3, 1.28, 1.12, 1.21, 1.05, 1.12, 1.4, 1.14],
                         [0.25, 0.2, 0.3, 0.12, 0.28, 0.05, 0.21, 0.14, 0.12, 0.13],
                         [1.75, 2.0, 2.3, 1.12, 0.5, 0.8, 0.1, 0.70, 1.12, 1.7],
                         [2.3, 1.8, 1.12, 0.8, 0.25, 1.2, 1.21, 1.14, 1.3, 1.25],
                         [1.05, 1.752, 0.8, 1.7, 1.3, 0.70, 2.3, 0.1, 1.12, 0.5],
                         [0.95, 1.02, 1.15, 1.77, 0.2, 1.38, 2.3, 0.1, 0.5, 0.70]]).T / 2.5
        if set(int(p) + 1 for p in oracle.reorder_perm(cols)[:3]) != {3, 5, 6}:
            return False
        # method vs definition on random data, all filters on
        Y = synth.uniform(800, 6, 3)
        ref = oracle.brute(Y, 0.35)
        if not np.array_equal(oracle.grid_join(Y, 0.35, 3), ref):
            return False
        # exact integer reference (independent of the oracle's loops)
        Z = synth.lattice(300, 5, seed=7, side=6)
        Zi = Z.astype(np.int64)
        dif = Zi[:, None, :] - Zi[None, :, :]
        want = np.argwhere((dif * dif).sum(-1) <= 3.0).astype(np.uint32)
        if not np.array_equal(oracle.grid_join(Z, math.sqrt(3.0) * (1 + 1e-12), 2), want):
            return False
        # Q join E against an integer reference, and its orientation
        Qz, Ez = synth.lattice(60, 4, seed=9, side=5), synth.lattice(90, 4, seed=10, side=5)
        dq = Qz.astype(np.int64)[:, None, :] - Ez.astype(np.int64)[None, :, :]
        wq = np.argwhere((dq * dq).sum(-1) <= 2).astype(np.uint32)
        if not np.array_equal(oracle.brute_qe(Qz, Ez, math.sqrt(2.0)), wq):
            return False
        # the boundary itself: eps = 2 is exact, pairs at distance 2 belong to R
        w4 = np.argwhere((dq * dq).sum(-1) <= 4).astype(np.uint32)
        if not np.array_equal(oracle.brute_qe(Qz, Ez, 2.0), w4):
            return False
        # one point's neighbours (the full-size tests' checker) on the lattice,
        # at an exact boundary (eps = 2) and away from the first row
        Xl = full_lattice(4, 3)
        for q in (0, 21, 42, 63):
            for eps, E in ((2.0, 4), (1.0, 1)):
                got = oracle.query_neighbors(Xl, eps, q).astype(np.int64)
                if not np.array_equal(got, lattice_row(Xl[q].astype(np.int64), 4, E)):
                    return False
        return True
    except (MemoryError, ValueError):
        return False


def test_real_oracle_passes_the_pins():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/present"
    msrc = tmp_path / "mut.c"
    msrc.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(msrc), "-lm"])
    saved_lib, saved_path = oracle._lib, oracle._LIB_PATH
    try:
        oracle._lib = None
        oracle._LIB_PATH = str(so)
        oracle._SRC_SAVED = oracle._SRC
        oracle._SRC = str(msrc)
        assert not _pins_pass(), f"mutant {name} slipped through the pins"
    finally:
        oracle._SRC = oracle._SRC_SAVED
        oracle._lib, oracle._LIB_PATH = saved_lib, saved_path


# ---------------------------------------------------------------------------
# constructNeighborTable (Python side of the oracle): mutants of the group-by
# ---------------------------------------------------------------------------

_real_table = oracle.neighbor_table


def _table_value_order_only(pairs, n):
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    order = np.argsort(p[:, 1], kind="stable")          # forgets the key
    counts = np.bincount(p[:, 0], minlength=n)
    rs = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rs[1:])
    return rs, p[order, 1].astype(np.uint32)


def _table_inclusive_starts(pairs, n):
    rs, nbr = _real_table(pairs, n)
    return np.concatenate([rs[1:], rs[-1:]]), nbr      # row a starts one row late


def _table_key_as_value(pairs, n):
    rs, _ = _real_table(pairs, n)
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    order = np.lexsort((p[:, 1], p[:, 0]))
    return rs, p[order, 0].astype(np.uint32)            # stores the key, not the value


@pytest.mark.parametrize("mutant", [_table_value_order_only, _table_inclusive_starts, _table_key_as_value])
def test_neighbor_table_pins_catch_mutants(mutant, monkeypatch):
    from tests import test_oracle_pins as pins
    pins.test_neighbor_table_rows_on_the_lattice(4, 3, 2)     # the real table passes
    monkeypatch.setattr(oracle, "neighbor_table", mutant)
    with pytest.raises(AssertionError):
        pins.test_neighbor_table_rows_on_the_lattice(4, 3, 2)
