"""CPU oracle for the ε-distance similarity self-join (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never does; the two share no
code.  The arithmetic lives in ``gj_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module compiles it with gcc on first use and
marshals numpy arrays into it.

Functions (paper section each follows):
  brute(X, eps)                     nested-loop join, the definition (Sec. 3.1)
  brute_qe(Q, E, eps)               the similarity join Q join_eps E by its definition (Sec. 3.1)
  grid_join(X, eps, k, ...)         the paper's method on the CPU (Sec. 3.2.1, 4.1–4.4, Alg. 1)
  query_neighbors(X, eps, q)        neighbours of one point by the definition
  variance / reorder_perm           REORDER (Sec. 4.2)
  cell_coords / linearise / adjacent_nonempty   grid index pieces (Sec. 3.2.1, Fig. 1)
  index_loss(n, k)                  l(n,k) of Sec. 4.1
  selectivity(R, n)                 S_D of Sec. 5.2
  depth_stats(X, eps, perm, qs)     SHORTC depth per candidate pair (Sec. 4.4)
  neighbor_table(pairs, n)          constructNeighborTable of Alg. 1 (Sec. 3.2.2) as CSR
Pairs are returned as an (m, 2) uint32 array sorted by (a, b).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gj_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

REORDER, SORTIDU, SHORTC = 1, 2, 4
ALL = REORDER | SORTIDU | SHORTC


class Stats(C.Structure):
    _fields_ = [("candidates", C.c_int64), ("window_candidates", C.c_int64),
                ("nonempty_cells", C.c_int64), ("k_used", C.c_int32),
                ("perm", C.c_int32 * 128)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction); returns the .so path."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-pthread", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        lib.gjo_sqdist.restype = C.c_double
        lib.gjo_sqdist.argtypes = [P, P, C.c_int]
        lib.gjo_brute.restype = C.c_int64
        lib.gjo_brute.argtypes = [P, C.c_int64, C.c_int, C.c_double, P, C.c_int64, C.c_int]
        lib.gjo_brute_qe.restype = C.c_int64
        lib.gjo_brute_qe.argtypes = [P, C.c_int64, P, C.c_int64, C.c_int, C.c_double, P, C.c_int64, C.c_int]
        lib.gjo_query_neighbors.restype = C.c_int64
        lib.gjo_query_neighbors.argtypes = [P, C.c_int64, C.c_int, C.c_double, C.c_int64,
                                            P, C.c_int64]
        lib.gjo_variance.restype = None
        lib.gjo_variance.argtypes = [P, C.c_int64, C.c_int, P, P]
        lib.gjo_reorder_perm.restype = None
        lib.gjo_reorder_perm.argtypes = [P, C.c_int, P]
        lib.gjo_index_loss.restype = C.c_double
        lib.gjo_index_loss.argtypes = [C.c_int, C.c_int]
        lib.gjo_cell_coords.restype = None
        lib.gjo_cell_coords.argtypes = [P, C.c_int64, C.c_int, C.c_int, P, P, P]
        lib.gjo_linearise.restype = C.c_int64
        lib.gjo_linearise.argtypes = [P, P, C.c_int]
        lib.gjo_adjacent_nonempty.restype = C.c_int
        lib.gjo_adjacent_nonempty.argtypes = [P, C.c_int64, P, P, C.c_int, P]
        lib.gjo_grid_join.restype = C.c_int64
        lib.gjo_grid_join.argtypes = [P, C.c_int64, C.c_int, C.c_double, C.c_int, C.c_int,
                                      C.c_int, P, C.c_int64, C.POINTER(Stats)]
        lib.gjo_depth_stats.restype = None
        lib.gjo_depth_stats.argtypes = [P, C.c_int64, C.c_int, C.c_double, P, P, C.c_int64,
                                        C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        _lib = lib
    return _lib


def _f64(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim != 2:
        raise ValueError("points must be an (n, d) array")
    return X


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def _keys_to_pairs(keys: np.ndarray) -> np.ndarray:
    out = np.empty((keys.size, 2), dtype=np.uint32)
    out[:, 0] = (keys >> np.uint64(32)).astype(np.uint32)
    out[:, 1] = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def _run_pairs(fn, expect_hint: int):
    cap = max(int(expect_hint), 1024)
    while True:
        buf = np.empty(cap, dtype=np.uint64)
        total = fn(buf, cap)
        if total < 0:
            raise MemoryError("oracle ran out of host memory" if total == -1 else "bad input")
        if total <= cap:
            return _keys_to_pairs(buf[:total])
        cap = int(total)


def sqdist(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return _load().gjo_sqdist(a.ctypes.data, b.ctypes.data, a.size)


def brute(X, eps: float, nthreads: int | None = None) -> np.ndarray:
    """All ordered pairs of R by the nested loop (Sec. 3.1)."""
    X = _f64(X)
    n, d = X.shape
    lib = _load()
    return _run_pairs(lambda buf, cap: lib.gjo_brute(X.ctypes.data, n, d, float(eps),
                                                     buf.ctypes.data, cap, _threads(nthreads)),
                      8 * n + 1024)


def brute_qe(Q, E, eps: float, nthreads: int | None = None) -> np.ndarray:
    """Q join_eps E (Sec. 3.1): every (q, e), q a row of Q and e a row of E,
    within eps, by the nested loop; sorted by (q, e)."""
    Q = _f64(Q)
    E = _f64(E)
    nq, d = Q.shape
    if E.shape[1] != d:
        raise ValueError("Q and E differ in dimension")
    ne = E.shape[0]
    lib = _load()
    return _run_pairs(lambda buf, cap: lib.gjo_brute_qe(Q.ctypes.data, nq, E.ctypes.data, ne, d, float(eps),
                                                        buf.ctypes.data, cap, _threads(nthreads)),
                      4 * (nq + ne) + 1024)


def brute_count(X, eps: float, nthreads: int | None = None) -> int:
    X = _f64(X)
    n, d = X.shape
    return int(_load().gjo_brute(X.ctypes.data, n, d, float(eps), None, 0, _threads(nthreads)))


def grid_join(X, eps: float, k: int, flags: int = ALL, nthreads: int | None = None,
              with_stats: bool = False):
    """R by the paper's method (REORDER / grid on k dims / SORTIDU / SHORTC)."""
    X = _f64(X)
    n, d = X.shape
    lib = _load()
    st = Stats()
    pairs = _run_pairs(lambda buf, cap: lib.gjo_grid_join(X.ctypes.data, n, d, float(eps), int(k),
                                                          int(flags), _threads(nthreads),
                                                          buf.ctypes.data, cap, C.byref(st)),
                       8 * n + 1024)
    if with_stats:
        return pairs, {"candidates": int(st.candidates),
                       "window_candidates": int(st.window_candidates),
                       "nonempty_cells": int(st.nonempty_cells),
                       "perm": [int(st.perm[j]) for j in range(min(d, 128))]}
    return pairs


def grid_count(X, eps: float, k: int, flags: int = ALL, nthreads: int | None = None) -> dict:
    """|R| and candidate counts by the paper's method, without keeping pairs."""
    X = _f64(X)
    n, d = X.shape
    st = Stats()
    total = _load().gjo_grid_join(X.ctypes.data, n, d, float(eps), int(k), int(flags),
                                  _threads(nthreads), None, 0, C.byref(st))
    if total < 0:
        raise MemoryError("oracle ran out of host memory" if total == -1 else "bad input")
    return {"R": int(total), "candidates": int(st.candidates),
            "window_candidates": int(st.window_candidates),
            "nonempty_cells": int(st.nonempty_cells)}


def query_neighbors(X, eps: float, q: int) -> np.ndarray:
    X = _f64(X)
    n, d = X.shape
    lib = _load()
    cnt = lib.gjo_query_neighbors(X.ctypes.data, n, d, float(eps), int(q), None, 0)
    out = np.empty(max(cnt, 1), dtype=np.uint32)
    lib.gjo_query_neighbors(X.ctypes.data, n, d, float(eps), int(q), out.ctypes.data, cnt)
    return out[:cnt]


def variance(X) -> tuple[np.ndarray, np.ndarray]:
    X = _f64(X)
    n, d = X.shape
    mean = np.empty(d)
    var = np.empty(d)
    _load().gjo_variance(X.ctypes.data, n, d, mean.ctypes.data, var.ctypes.data)
    return mean, var


def reorder_perm(X) -> np.ndarray:
    """REORDER permutation: dimension indices by descending variance (Sec. 4.2)."""
    _, var = variance(X)
    perm = np.empty(var.size, dtype=np.int32)
    _load().gjo_reorder_perm(var.ctypes.data, var.size, perm.ctypes.data)
    return perm


def index_loss(n: int, k: int) -> float:
    return float(_load().gjo_index_loss(int(n), int(k)))


def cell_coords(Y, k: int, origin, width) -> np.ndarray:
    Y = _f64(Y)
    n, d = Y.shape
    origin = np.ascontiguousarray(origin, dtype=np.float64)
    width = np.ascontiguousarray(np.broadcast_to(width, (k,)), dtype=np.float64)
    out = np.empty((n, max(k, 1)), dtype=np.int64)
    _load().gjo_cell_coords(Y.ctypes.data, n, d, int(k), origin.ctypes.data, width.ctypes.data,
                            out.ctypes.data)
    return out[:, :k]


def linearise(coord, ncells) -> int:
    c = np.ascontiguousarray(coord, dtype=np.int64)
    nc = np.ascontiguousarray(ncells, dtype=np.int64)
    return int(_load().gjo_linearise(c.ctypes.data, nc.ctypes.data, c.size))


def adjacent_nonempty(ids_sorted, coord, ncells) -> np.ndarray:
    ids = np.ascontiguousarray(ids_sorted, dtype=np.int64)
    c = np.ascontiguousarray(coord, dtype=np.int64)
    nc = np.ascontiguousarray(ncells, dtype=np.int64)
    out = np.empty(3 ** c.size, dtype=np.int64)
    m = _load().gjo_adjacent_nonempty(ids.ctypes.data, ids.size, c.ctypes.data, nc.ctypes.data,
                                      c.size, out.ctypes.data)
    return out[:m]


def selectivity(R: int, n: int) -> float:
    """S_D = (|R| - |D|) / |D| (Sec. 5.2)."""
    return (R - n) / n


def depth_stats(X, eps: float, perm, queries, nthreads: int | None = None) -> tuple[int, int]:
    """(Σ SHORTC depth, pair count) over every (q, j≠q) for the listed queries,
    dimensions taken in the order ``perm`` (Sec. 4.4)."""
    X = _f64(X)
    n, d = X.shape
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    qs = np.ascontiguousarray(queries, dtype=np.int64)
    ds, pc = C.c_int64(), C.c_int64()
    _load().gjo_depth_stats(X.ctypes.data, n, d, float(eps), perm.ctypes.data, qs.ctypes.data,
                            qs.size, _threads(nthreads), C.byref(ds), C.byref(pc))
    return int(ds.value), int(pc.value)


def neighbor_table(pairs, n: int) -> tuple[np.ndarray, np.ndarray]:
    """constructNeighborTable (Alg. 1; Sec. 3.2.2): the key/value result pairs
    stored with each key once.  As compressed sparse rows over the point order:
    the neighbours of a are nbr[row_start[a]:row_start[a+1]], ascending.
    A plain group-by: sort the pairs by (key, value), count the keys."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    order = np.lexsort((p[:, 1], p[:, 0]))
    nbr = p[order, 1].astype(np.uint32)
    counts = np.bincount(p[:, 0], minlength=n) if p.size else np.zeros(n, dtype=np.int64)
    row_start = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_start[1:])
    return row_start, nbr
