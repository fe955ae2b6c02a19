"""The tensor-core filter's survivor threshold T against an emulation of its
arithmetic, on the CPU (no device needed).

The filter keeps a pair iff t <= T, with t = |h_a|^2 + |h_b|^2 - 2 <h_a, h_b>
formed from fp16 coordinates h = rn16(sigma (x - c)) as one K-term dot
product of fp16 operands with fp32 accumulation: A row [-2h, |h|^2_hi,
|h|^2_lo, 1, 1], B row [h, 1, 1, |h|^2_hi, |h|^2_lo]. The library's T must
cover every pair within eps for any accumulation order. Here the products are
formed exactly (fp16 x fp16 fits in fp32), and the fp32 sums are taken in
several orders, including a truncating (round-toward-zero) adder. Every pair
with FP64 squared distance <= eps^2 must give t <= T in each of them. The
T used is the library's own (gj_tc_threshold), not a re-derivation.
"""
import numpy as np
import pytest

import synth

gj = pytest.importorskip("paper_1809_09930_gb300.gj")


def _scale(X):
    """Centre (per-dimension midrange), radius bound R0 and power-of-two scale
    sigma, as the tensor-core form chooses them."""
    c = 0.5 * (X.min(axis=0) + X.max(axis=0))
    R0 = float(np.sqrt(((X - c) ** 2).sum(axis=1).max())) * (1 + 2.0 ** -30)
    sigma = 2.0 ** np.floor(np.log2(250.0 / R0))
    return c, R0, sigma


def _operands(X, c, sigma):
    """fp16 operand rows as float64 arrays (exact values)."""
    h = ((X - c) * sigma).astype(np.float16).astype(np.float64)
    nrm = np.zeros(len(X))
    for j in range(X.shape[1]):   # FP64 sum of the squares, dimension order
        nrm = nrm + h[:, j] * h[:, j]
    hi = nrm.astype(np.float16).astype(np.float64)
    lo = (nrm - hi).astype(np.float16).astype(np.float64)
    one = np.ones(len(X))
    A = np.column_stack([-2.0 * h, hi, lo, one, one])
    B = np.column_stack([h, one, one, hi, lo])
    return A, B


def _add_rz(a, b):
    """fp32 a + b rounded toward zero (a truncating adder); the fp64 sum of two
    fp32 values is exact here (their exponents differ by far less than 29)."""
    z = a.astype(np.float64) + b.astype(np.float64)
    r = z.astype(np.float32)
    over = np.abs(r.astype(np.float64)) > np.abs(z)
    r[over] = np.nextafter(r[over], np.float32(0.0))
    return r


def _accumulate(P, order, mode):
    """Sum the K product columns of P (pairs x K, exact fp32 values) in fp32."""
    acc = np.zeros(P.shape[0], dtype=np.float32)
    if mode == "tree":
        cols = [P[:, k].astype(np.float32) for k in order]
        while len(cols) > 1:
            nxt = [cols[i] + cols[i + 1] for i in range(0, len(cols) - 1, 2)]
            if len(cols) % 2:
                nxt.append(cols[-1])
            cols = nxt
        return cols[0]
    for k in order:
        col = P[:, k].astype(np.float32)
        acc = _add_rz(acc, col) if mode == "rz" else (acc + col).astype(np.float32)
    return acc


def _pairs_within(X, eps):
    """All pairs i < j (and the self-pairs) with FP64 squared distance <= eps^2."""
    n = len(X)
    i, j = np.triu_indices(n)
    s = ((X[i] - X[j]) ** 2).sum(axis=1)
    keep = s <= eps * eps
    return i[keep], j[keep]


def _boundary_points(X, eps, c, rng, m):
    """Pairs built at distance just inside eps, anchored at the points farthest
    from the centre (where the fp16 rounding errs the most)."""
    far = np.argsort(-((X - c) ** 2).sum(axis=1))[:m]
    u = rng.standard_normal((m, X.shape[1]))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Y = X[far] + eps * (1 - 1e-12) * u
    return np.vstack([X, Y])


@pytest.mark.parametrize("kind,n,d,frac", [
    ("uniform", 700, 3, 0.2),
    ("uniform", 600, 16, 0.3),
    ("mixture", 600, 32, 0.1),
    ("skewed", 500, 18, 0.05),
    ("exponential", 500, 64, 0.05),
    ("uniform", 300, 124, 0.3),
])
def test_every_pair_within_eps_survives_in_any_accumulation_order(kind, n, d, frac):
    rng = np.random.default_rng(n * 131 + d)
    X = synth.generate(kind, n, d, seed=d + 7)
    # eps at the frac quantile of the pair distances, so that many pairs lie near it
    ii, jj = np.triu_indices(len(X), 1)
    sel = rng.choice(len(ii), size=min(len(ii), 20000), replace=False)
    eps = float(np.quantile(np.sqrt(((X[ii[sel]] - X[jj[sel]]) ** 2).sum(axis=1)), frac))
    c, _, _ = _scale(X)
    X = _boundary_points(X, eps, c, rng, 64)
    c, R0, sigma = _scale(X)
    st, T = gj.gj_tc_threshold(eps, sigma, R0, d)
    assert st == gj.GJ_OK
    A, B = _operands(X, c, sigma)
    i, j = _pairs_within(X, eps)
    assert len(i) > len(X)   # more than the self-pairs
    P = A[i] * B[j]          # exact: fp16 x fp16 products need 22 bits
    assert np.all(P.astype(np.float32).astype(np.float64) == P)
    K = P.shape[1]
    orders = {"sequential": list(range(K)), "reversed": list(range(K))[::-1],
              "norms first": list(range(d, K)) + list(range(d)),
              "random": list(rng.permutation(K))}
    Tf = np.float32(T)
    # the boundary pairs do exceed (sigma eps)^2 in the emulation, so a
    # threshold without a margin would fail this test
    t0 = _accumulate(P, orders["sequential"], "rn")
    assert np.any(t0.astype(np.float64) > (sigma * eps) ** 2)
    for name, order in orders.items():
        for mode in ("rn", "rz"):
            t = _accumulate(P, order, mode)
            worst = int(np.argmax(t))
            assert np.all(t <= Tf), (name, mode, float(t[worst]), float(Tf))
    t = _accumulate(P, list(range(K)), "tree")
    assert np.all(t <= Tf)


def test_threshold_is_tight_for_moderate_eps():
    """The margin adds a few percent, not more, when sigma*eps is large beside
    the fp16 rounding (the survivor count stays near |R|)."""
    X = synth.uniform(2000, 16, 3)
    c, R0, sigma = _scale(X)
    st, T = gj.gj_tc_threshold(0.3, sigma, R0, 16)
    assert st == gj.GJ_OK
    se2 = (sigma * 0.3) ** 2
    assert se2 < T < 1.05 * se2


def test_threshold_argument_checks():
    assert gj.gj_tc_threshold(0.0, 1.0, 1.0, 16)[0] == gj.GJ_ERR_INVALID_ARG
    assert gj.gj_tc_threshold(0.1, -1.0, 1.0, 16)[0] == gj.GJ_ERR_INVALID_ARG
    assert gj.gj_tc_threshold(0.1, 1.0, float("nan"), 16)[0] == gj.GJ_ERR_INVALID_ARG
    assert gj.gj_tc_threshold(0.1, 1.0, 1.0, 0)[0] == gj.GJ_ERR_INVALID_ARG
    assert gj.gj_tc_threshold(0.1, 1.0, 1.0, 125)[0] == gj.GJ_ERR_INVALID_ARG
    assert gj.gj_tc_threshold(0.1, 1.0, 1.0, 124)[0] == gj.GJ_OK


def test_qe_packing_covers_queries_beyond_the_entries():
    """Q join_eps E packs queries and entries under the entries' centre with one
    scale and one radius bound taken over both sets.  Queries a full eps
    outside the entries' ball, each with a partner just inside eps: every
    query-entry pair within eps must give t <= T in any accumulation order.
    With the entries' own scale and radius the same pairs fail (the query
    norms overflow fp16, or exceed the margin), so the wider choice is needed."""
    rng = np.random.default_rng(17)
    d = 16
    E = synth.uniform(600, d, 5)
    c, R0e, sigma_e = _scale(E)
    eps = 0.6 * R0e
    far = np.argsort(-((E - c) ** 2).sum(axis=1))[:150]
    out = (E[far] - c) / np.linalg.norm(E[far] - c, axis=1, keepdims=True)
    jitter = rng.standard_normal((150, d)) * 0.05
    u = out + jitter
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Q = np.vstack([E[far] + eps * (1 - 1e-12) * u, synth.uniform(100, d, 6)])
    R0q = float(np.sqrt(((Q - c) ** 2).sum(axis=1).max())) * (1 + 2.0 ** -30)
    assert R0q > R0e * 1.4
    R0 = max(R0e, R0q)
    sigma = 2.0 ** np.floor(np.log2(250.0 / R0))
    s = ((Q[:, None, :] - E[None, :, :]) ** 2).sum(axis=2)
    i, j = np.nonzero(s <= eps * eps)
    assert len(i) >= 150
    st, T = gj.gj_tc_threshold(eps, sigma, R0, d)
    assert st == gj.GJ_OK
    A, _ = _operands(Q, c, sigma)
    _, B = _operands(E, c, sigma)
    P = A[i] * B[j]
    assert np.all(P.astype(np.float32).astype(np.float64) == P)
    K = P.shape[1]
    Tf = np.float32(T)
    for order in (list(range(K)), list(range(K))[::-1], list(range(d, K)) + list(range(d))):
        for mode in ("rn", "rz"):
            assert np.all(_accumulate(P, order, mode) <= Tf)
    assert np.all(_accumulate(P, list(range(K)), "tree") <= Tf)
    # the entries' own packing loses pairs
    st, Te = gj.gj_tc_threshold(eps, sigma_e, R0e, d)
    assert st == gj.GJ_OK
    with np.errstate(over="ignore", invalid="ignore"):
        Ae, _ = _operands(Q, c, sigma_e)
        _, Be = _operands(E, c, sigma_e)
        te = _accumulate(Ae[i] * Be[j], list(range(K)), "rn")
    assert not np.all(te <= np.float32(Te))
