"""Comparison of a GPU pair set with the oracle's, under the tie rule.

The GPU sums squared differences in REORDER order with fused multiply-add;
the oracle sums in the original order without.  Both are exact FP64 results of
their own order, so the two sets may differ only on pairs whose squared
distance lies within 1e-12 relative of fl(eps^2) (the admissible tie band).
Every such pair is listed; any other difference fails.
"""
from __future__ import annotations

import numpy as np

import oracle

TIE_REL = 1e-12


def keys(p: np.ndarray) -> np.ndarray:
    p = np.asarray(p, dtype=np.uint64).reshape(-1, 2)
    return np.sort((p[:, 0] << np.uint64(32)) | p[:, 1])


def compare(X: np.ndarray, eps: float, gpu_pairs: np.ndarray, ref_pairs: np.ndarray) -> dict:
    g = keys(gpu_pairs)
    r = keys(ref_pairs)
    assert np.all(np.diff(g.astype(np.int64)) != 0) or g.size < 2, "duplicate pairs in GPU output"
    missing = np.setdiff1d(r, g, assume_unique=True)
    extra = np.setdiff1d(g, r, assume_unique=True)
    e2 = eps * eps
    ties = []
    bad = []
    for k in np.concatenate([missing, extra]):
        a, b = int(k >> np.uint64(32)), int(k & np.uint64(0xFFFFFFFF))
        s = oracle.sqdist(X[a], X[b])
        (ties if abs(s - e2) <= TIE_REL * e2 else bad).append((a, b, s))
    return {"gpu": int(g.size), "ref": int(r.size), "missing": int(missing.size),
            "extra": int(extra.size), "ties": ties, "bad": bad}


def assert_parity(X, eps, gpu_pairs, ref_pairs):
    res = compare(X, eps, gpu_pairs, ref_pairs)
    assert not res["bad"], f"pairs outside the tie band differ: {res['bad'][:5]} ({res})"
    return res
