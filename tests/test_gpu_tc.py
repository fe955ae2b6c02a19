"""Tensor-core filter (GJ_TC_FILTER): layout, error model, exactness.

The filter only decides which candidates reach the FP64 recheck, and the
recheck is the plain path's own arithmetic, so the TC path must return exactly
the plain path's pair set (not merely the same set up to ties), and that set
must match the oracle up to the tie band.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.parity import assert_parity, keys

pytestmark = pytest.mark.gpu

gj = pytest.importorskip("paper_1809_09930_gb300.gj")

TC = gj.GJ_DEFAULT_FLAGS | gj.GJ_TC_FILTER


def _rand_f16(shape, seed, scale=1.0):
    u = synth.uniform01(seed, int(np.prod(shape))).reshape(shape)
    return ((u * 2.0 - 1.0) * scale).astype(np.float16)


def _adversarial_tile(Kp, variant, seed):
    """A, B (fp16, 128 x Kp) whose fp32 sums are hard to get right.
    cancel: per row two products +-250*250 at row-dependent K positions (the
      large pair falls early, late or in the middle of the sum), every other
      product 250 * (r 2^-17), an fp16 subnormal times 250, just below half an
      fp32 ulp of 62500: added beside the large terms they round away; B's
      signs random, so about half the entries cancel to the small terms.
    same-sign: as cancel with both large products positive.
    norms: the filter's own rows, A = [-2h, |h|^2_hi, |h|^2_lo, 1, 1] and
      B = [h', 1, 1, |h'|^2_hi, |h'|^2_lo] with |h| near 250 and h' = h plus a
      small offset: terms of 62500 cancel down to a small |h - h'|^2."""
    rng = np.random.default_rng(seed)
    A = np.zeros((128, Kp), dtype=np.float64)
    B = np.zeros((128, Kp), dtype=np.float64)
    if variant in ("cancel", "same-sign"):
        r = rng.integers(8, 16, size=(128, Kp)) / 16.0
        A[:] = r * 2.0 ** -17
        for i in range(128):
            k1 = i % Kp
            k2 = (i * 7 + 3) % Kp
            if k2 == k1:
                k2 = (k1 + 1) % Kp
            A[i, k1] = 250.0
            A[i, k2] = -250.0 if variant == "cancel" else 250.0
        B[:] = 250.0
        if variant == "cancel":
            B[rng.random((128, Kp)) < 0.5] *= -1.0
    else:
        d = Kp - 4

        def rows(n, base=None):
            if base is None:
                h = rng.normal(size=(n, d))
                h *= (250.0 * rng.uniform(0.97, 1.0, size=(n, 1))) / np.linalg.norm(h, axis=1, keepdims=True)
            else:
                h = base + rng.normal(scale=0.05, size=base.shape)
            # magnitudes >= 1/4 keep every product a multiple of 2^-24 and the
            # fp64 reference sums exact (at most 42 significant bits)
            h = np.where(h < 0, -1.0, 1.0) * np.maximum(np.abs(h), 0.25)
            h = h.astype(np.float16).astype(np.float64)
            nrm = (h * h).sum(axis=1)
            hi = nrm.astype(np.float16).astype(np.float64)
            lo = (nrm - hi).astype(np.float16).astype(np.float64)
            return h, hi, lo

        ha, hia, loa = rows(128)
        hb, hib, lob = rows(128, ha)
        A[:, :d] = -2.0 * ha
        A[:, d], A[:, d + 1], A[:, d + 2], A[:, d + 3] = hia, loa, 1.0, 1.0
        B[:, :d] = hb
        B[:, d], B[:, d + 1], B[:, d + 2], B[:, d + 3] = 1.0, 1.0, hib, lob
    return A.astype(np.float16), B.astype(np.float16)


@pytest.mark.parametrize("Kp", [16, 48, 128])
@pytest.mark.parametrize("variant", ["cancel", "same-sign", "norms"])
def test_single_tile_adversarial_accumulation(Kp, variant):
    """The accumulation model where it is tightest: exact fp16 products (their
    fp64 sums are exact here), fp32 results within (Kp + 2) 2^-22 of the sum
    of |terms| on every entry."""
    A, B = _adversarial_tile(Kp, variant, 300 + Kp)
    D = gj.gj_debug_tc_tile(A, B).astype(np.float64)
    a = A.astype(np.float64)
    b = B.astype(np.float64)
    exact = a @ b.T
    absum = np.abs(a) @ np.abs(b).T
    bound = (Kp + 2) * 2.0 ** -22 * absum
    ratio = np.abs(D - exact) / bound
    print(f"Kp={Kp} {variant}: worst err/bound {ratio.max():.4f}, worst |err| {np.abs(D - exact).max():.3g}")
    assert np.all(ratio <= 1.0), f"worst err/bound {ratio.max()}"


def test_planted_pairs_at_the_largest_radius_d124():
    """Pairs at eps (1 - 2^-40) on a sphere of the largest radius about the
    filter's centre (points mirrored through the origin, so the per-dimension
    midrange is 0), d = 124, Kp = 128: the filter's margin is dominated by its
    accumulation term there.  Every planted pair within eps must be found."""
    d, m, rho, eps = 124, 1500, 40.0, 0.05
    u = synth.normal(501, m * d).reshape(m, d)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = synth.normal(502, m * d).reshape(m, d)
    v -= (v * u).sum(axis=1, keepdims=True) * u          # orthogonal to u: the partner stays near radius rho
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    base = rho * u
    partner = base + v * (eps * (1.0 - 2.0 ** -40))
    X = np.vstack([base, partner, -base, -partner])
    plain, tc, st = _both(X, eps, k=1)
    assert np.array_equal(keys(plain), keys(tc))
    got = set(keys(tc).tolist())
    found = inside = 0
    for off in (0, 2 * m):
        for i in range(m):
            a, b = off + i, off + m + i
            if oracle.sqdist(X[a], X[b]) <= eps * eps:
                inside += 1
                found += ((a << 32) | b) in got and ((b << 32) | a) in got
    assert found == inside and inside > 0.8 * 2 * m


@pytest.mark.parametrize("Kp", [16, 32, 48, 96, 128])
def test_single_tile_layout_and_error_model(Kp):
    A = _rand_f16((128, Kp), 100 + Kp, 40.0)
    B = _rand_f16((128, Kp), 200 + Kp, 40.0)
    D = gj.gj_debug_tc_tile(A, B)
    a = A.astype(np.float64)
    b = B.astype(np.float64)
    exact = a @ b.T                       # products of fp16 values are exact in fp64
    absum = np.abs(a) @ np.abs(b).T
    err = np.abs(D.astype(np.float64) - exact)
    bound = (Kp + 2) * 2.0 ** -22 * absum  # the filter's accumulation model
    assert np.all(err <= bound), f"max err/bound = {np.max(err / np.maximum(bound, 1e-300))}"
    # the layout is right only if every entry is close (a wrong row/K mapping is O(1) off)
    assert np.max(err / np.maximum(absum, 1e-30)) < 1e-5


def test_single_tile_structured_rows_and_columns():
    """One-hot rows expose any row, column or K-chunk mix-up."""
    Kp = 64
    A = np.zeros((128, Kp), dtype=np.float16)
    B = np.zeros((128, Kp), dtype=np.float16)
    for i in range(128):
        A[i, i % Kp] = 1.0
        A[i, (i * 7 + 3) % Kp] += np.float16(i / 128.0)
        B[i, (i * 5 + 1) % Kp] = np.float16((i + 1) / 64.0)
    D = gj.gj_debug_tc_tile(A, B)
    assert np.array_equal(D, (A.astype(np.float32) @ B.astype(np.float32).T))


def _both(X, eps, k=0, **kw):
    with gj.Index(X, eps, k=k, **kw) as ip:
        plain = ip.join()
    with gj.Index(X, eps, k=k, flags=TC, **kw) as it:
        tc = it.join()
        st = it.stats()
    return plain, tc, st


@pytest.mark.parametrize("kind,n,d,eps,k", [
    ("uniform", 3001, 16, 0.9, 0),
    ("uniform", 2500, 32, 1.3, 0),
    ("uniform", 1800, 64, 2.3, 1),
    ("mixture", 5000, 32, 0.33, 3),
    ("skewed", 7000, 18, 0.12, 3),
    ("mixture", 1500, 90, 0.56, 2),
    ("uniform", 5000, 3, 0.05, 3),
    ("exponential", 3000, 16, 0.06, 2),
])
def test_tc_equals_plain_and_oracle(kind, n, d, eps, k):
    X = synth.generate(kind, n, d, seed=n + 3 * d)
    plain, tc, st = _both(X, eps, k=k)
    assert np.array_equal(keys(plain), keys(tc)), "TC path differs from the plain path"
    assert st["tc_survivors"] >= (len(tc) + n) // 2   # every unordered pair of R survived the filter
    ref = oracle.brute(X, eps)
    assert_parity(X, eps, tc, ref)


def test_adversarial_pairs_at_the_boundary_far_from_the_centre():
    """Pairs at distance eps*(1 - 1e-9) placed where |x - c| is large relative
    to eps (the filter's margin is smallest relative to its error there)."""
    d, eps = 32, 0.05
    base = synth.uniform(600, d, 77) * 40.0            # wide spread: R0 >> eps
    dirs = synth.normal(78, 600 * d).reshape(600, d)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    partner = base + dirs * eps * (1.0 - 1e-9)
    X = np.vstack([base, partner])
    plain, tc, st = _both(X, eps, k=1)
    assert np.array_equal(keys(plain), keys(tc))
    ref = oracle.brute(X, eps)
    assert_parity(X, eps, tc, ref)
    got = set(keys(tc).tolist())
    n0 = 600
    found = sum(1 for i in range(n0) if ((i << 32) | (i + n0)) in got)
    # the partner lies inside eps up to FP64 rounding of the construction
    inside = sum(1 for i in range(n0) if oracle.sqdist(X[i], X[i + n0]) <= eps * eps)
    assert found == inside and inside > 550


def test_tc_lattice_exact():
    X = synth.lattice(3000, 8, seed=5, side=4)
    for eps in (1.0, math.sqrt(2.0), 2.0):
        ref = oracle.brute(X, eps)
        with gj.Index(X, eps, k=2, flags=TC) as ix:
            got = ix.join()
        assert np.array_equal(keys(got), keys(ref))


def test_tc_small_batches_resume_exactly():
    X = synth.mixture(8000, 18, 6)
    ref = oracle.brute(X, 0.35)
    with gj.Index(X, 0.35, k=2, flags=TC | gj.GJ_HOST_BATCHED, batch_pairs=150_000) as ix:
        got = ix.join()
        st = ix.stats()
    assert st["launches"] > 3     # result batches of 150,000 pairs, each resumed exactly
    assert_parity(X, 0.35, got, ref)


def test_tc_capacity_count_and_device_output():
    torch = pytest.importorskip("torch")
    X = synth.uniform(6000, 16, 14)
    ref = oracle.brute(X, 0.8)
    with gj.Index(X, 0.8, k=0, flags=TC) as ix:
        assert ix.count() == len(ref)
        small = np.empty((len(ref) // 4, 2), dtype=np.uint32)
        st, n = gj.gj_self_join(ix.h, small)
        assert st == gj.GJ_ERR_CAPACITY and n == len(ref)
        out = torch.empty((len(ref), 2), dtype=torch.int32, device="cuda")
        st, n = gj.gj_self_join(ix.h, out)
        assert st == gj.GJ_OK and n == len(ref)
        got = out.cpu().numpy().view(np.uint32)
    assert_parity(X, 0.8, got, ref)


def test_tc_duplicates_dense_output():
    """All points equal: every slot of every tile is a result pair, the largest
    output a tile can produce (exercises staging flushes)."""
    X = np.full((3000, 16), 0.25)
    with gj.Index(X, 1e-3, k=1, flags=TC) as ix:
        n = ix.count()
        assert n == 3000 * 3000
        got = ix.join()
    assert len(np.unique(keys(got))) == 3000 * 3000


def test_tc_entity_partitions():
    X = synth.uniform(9000, 32, 19)
    ref = oracle.brute(X, 1.25)
    with gj.Index(X, 1.25, k=0, flags=TC) as ix:
        parts = [ix.join(part=p, nparts=3) for p in range(3)]
    allp = np.concatenate(parts)
    assert len(np.unique(keys(allp))) == len(allp)
    assert_parity(X, 1.25, allp, ref)
