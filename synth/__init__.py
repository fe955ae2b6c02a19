"""Seeded synthetic point sets for the ε-distance self-join.

This module only draws random numbers and shapes them into point sets; it holds
none of the join's arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA
library are fed from here, so that the two see the same bytes.

Every value comes from the splitmix64 generator (Steele, Lea & Flood 2014):
stream element ``i`` of seed ``s`` is ``mix(s + (i+1)·0x9E3779B97F4A7C15)`` with
the published 64-bit finaliser.  Doubles take the top 53 bits
(``(z >> 11)·2⁻⁵³``, uniform in [0,1)); normals use Box–Muller on two uniforms.
Sub-streams (cluster centres, widths, labels, coordinates) use derived seeds so
that changing one shape parameter does not shift the others.

Workload shapes follow the paper's synthetic and real workloads (Table 1:
16–90 dimensions, 6.8e4–5e6 points; Sec. 5.1 "Syn-" data) as restated in the
project's configuration list:

* ``uniform``   — i.i.d. U[0,1)^d (the tiny and paper-scale configurations).
* ``mixture``   — 64 isotropic Gaussian clusters (σ = 0.05, centres U[0,1)^d)
  plus 10 % uniform background (stand-in for the 32-D image-feature sets and
  the 90-D song features, which are not available here).
* ``skewed``    — 10 anisotropic Gaussian clusters with per-dimension σ
  log-uniform in [0.01, 0.2], 90 % of points, plus 10 % uniform (stand-in for
  the 18-D particle-physics set).
* ``exponential`` — the paper's own "Syn-" data: i.i.d. exponential with
  λ = 40, clipped into [0,1] (Sec. 5.1).
* ``lattice``   — small integers, for exact-arithmetic boundary tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _C1
    z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def derive_seed(seed: int, stream: int) -> int:
    """A seed for sub-stream ``stream`` of ``seed`` (one splitmix64 step)."""
    z = np.array([(int(seed) + (int(stream) + 1) * 0x9E3779B97F4A7C15) & (2**64 - 1)],
                 dtype=np.uint64)
    return int(_mix(z)[0])


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Elements ``offset .. offset+count-1`` of the splitmix64 stream of ``seed``."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(int(seed) & (2**64 - 1))
    for lo in range(0, count, _CHUNK):
        hi = min(count, lo + _CHUNK)
        idx = np.arange(offset + lo + 1, offset + hi + 1, dtype=np.uint64)
        out[lo:hi] = _mix(s + idx * _GAMMA)
    return out


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles uniform in [0,1) (53-bit)."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box–Muller (cosine branch only)."""
    z = splitmix64(seed, 2 * count)
    u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0,1]
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)          # [0,1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def uniform(n: int, d: int, seed: int) -> np.ndarray:
    """n×d row-major points, i.i.d. U[0,1)."""
    return uniform01(seed, n * d).reshape(n, d)


def mixture(n: int, d: int, seed: int, clusters: int = 64, sigma: float = 0.05,
            background: float = 0.10) -> np.ndarray:
    """Isotropic Gaussian mixture plus a uniform background fraction."""
    centres = uniform(clusters, d, derive_seed(seed, 1))
    lab_u = uniform01(derive_seed(seed, 2), n)
    which = np.minimum((uniform01(derive_seed(seed, 3), n) * clusters).astype(np.int64),
                       clusters - 1)
    g = normal(derive_seed(seed, 4), n * d).reshape(n, d)
    x = centres[which] + sigma * g
    bg = lab_u < background
    nbg = int(bg.sum())
    if nbg:
        x[bg] = uniform(nbg, d, derive_seed(seed, 5))
    return np.ascontiguousarray(x)


def skewed(n: int, d: int, seed: int, clusters: int = 10, sigma_lo: float = 0.01,
           sigma_hi: float = 0.2, background: float = 0.10) -> np.ndarray:
    """Anisotropic Gaussian clusters (σ per cluster and dimension log-uniform in
    [sigma_lo, sigma_hi]) holding 1-background of the points, plus uniform background."""
    centres = uniform(clusters, d, derive_seed(seed, 11))
    lu = uniform(clusters, d, derive_seed(seed, 12))
    sig = np.exp(math.log(sigma_lo) + lu * (math.log(sigma_hi) - math.log(sigma_lo)))
    lab_u = uniform01(derive_seed(seed, 13), n)
    which = np.minimum((uniform01(derive_seed(seed, 14), n) * clusters).astype(np.int64),
                       clusters - 1)
    g = normal(derive_seed(seed, 15), n * d).reshape(n, d)
    x = centres[which] + sig[which] * g
    bg = lab_u < background
    nbg = int(bg.sum())
    if nbg:
        x[bg] = uniform(nbg, d, derive_seed(seed, 16))
    return np.ascontiguousarray(x)


def exponential(n: int, d: int, seed: int, lam: float = 40.0) -> np.ndarray:
    """The paper's Syn- data: i.i.d. exponential(λ) clipped into [0,1] (Sec. 5.1)."""
    u = ((splitmix64(seed, n * d) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    return np.minimum(-np.log(u) / lam, 1.0).reshape(n, d)


def lattice(n: int, d: int, seed: int, side: int = 4) -> np.ndarray:
    """Integer lattice points in [0, side)^d (exact in any summation order)."""
    z = splitmix64(seed, n * d)
    return (z % np.uint64(side)).astype(np.float64).reshape(n, d)


def generate(kind: str, n: int, d: int, seed: int) -> np.ndarray:
    if kind == "uniform":
        return uniform(n, d, seed)
    if kind == "mixture":
        return mixture(n, d, seed)
    if kind == "skewed":
        return skewed(n, d, seed)
    if kind == "exponential":
        return exponential(n, d, seed)
    if kind == "lattice":
        return lattice(n, d, seed)
    raise ValueError(f"unknown point-set kind {kind!r}")


@dataclass(frozen=True)
class JobSpec:
    """One independent self-join of the many-jobs workload."""
    n: int
    d: int
    kind: str
    seed: int
    target_nb: float   # mean neighbours the job's ε is chosen for


def many_jobs(count: int = 256, seed: int = 4, n_lo: int = 1000, n_hi: int = 200_000,
              dims=(16, 18, 32), nb_lo: float = 8.0, nb_hi: float = 128.0) -> list[JobSpec]:
    """The uneven-jobs workload: n log-uniform in [n_lo, n_hi], d cycling over
    ``dims`` at random, uniform and mixture data alternating, target mean
    neighbours log-uniform in [nb_lo, nb_hi]."""
    u = uniform(count, 3, derive_seed(seed, 21))
    jobs = []
    for j in range(count):
        n = int(round(math.exp(math.log(n_lo) + u[j, 0] * (math.log(n_hi) - math.log(n_lo)))))
        d = dims[min(int(u[j, 1] * len(dims)), len(dims) - 1)]
        nb = math.exp(math.log(nb_lo) + u[j, 2] * (math.log(nb_hi) - math.log(nb_lo)))
        kind = "uniform" if j % 2 == 0 else "mixture"
        jobs.append(JobSpec(n=n, d=d, kind=kind, seed=derive_seed(seed, 1000 + j), target_nb=nb))
    return jobs
