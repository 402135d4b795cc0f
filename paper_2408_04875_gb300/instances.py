"""Seeded synthetic UBQP instances shaped like the paper's workloads.

This module only draws numbers: it holds none of the method's arithmetic, so both
the CUDA library's callers and the FP64 oracle's tests may use it.  Every random
quantity the method consumes (the symmetric perturbation mu of Sec. 3.6 and the
extra starting points of a restart batch) is drawn here and passed in as an input.

Families (value ranges follow Sec. 5: random instances, BE ranges, rudy/G-set
Max-Cut graphs with +-1 weights):

* ``random_ubqp``  - upper triangle incl. diagonal kept with probability
  ``density``, integer values uniform in [lo, hi], mirrored; b = 0 or integers.
* ``maxcut_ubqp``  - G(n, density) with +-1 edge weights W, mapped to the 0/1
  form f(y) = y^T W y - (W e)^T y = -cut(y)  (the Max-Cut model of Sec. 5.3).
* ``perturbation`` - symmetric N(0, sigma) on the stored entries of Q (Sec. 3.6).

Streams: every draw uses numpy.random.Generator(PCG64(SeedSequence(key))) with a
key built from (family tag, n, seed), so instances never share a stream.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng_for", "random_ubqp", "dense_ubqp", "maxcut_ubqp", "perturbation",
    "random_starts", "box_points", "c1_instance", "c2_instance", "c3_instance",
    "c4_instance", "c5_specs", "c5_instance",
]

_TAG_RANDOM, _TAG_DENSE, _TAG_MAXCUT, _TAG_MU, _TAG_STARTS, _TAG_BOX, _TAG_C5 = range(1, 8)


def rng_for(*key: int) -> np.random.Generator:
    """PCG64 generator keyed by a tuple of non-negative integers."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


def _mirror_upper(U: np.ndarray) -> np.ndarray:
    """Symmetric matrix from an upper triangle (diagonal kept once)."""
    return np.triu(U) + np.triu(U, 1).T


def random_ubqp(n: int, density: float, seed: int, lo: int = -100, hi: int = 100,
                b_range: tuple[int, int] | None = None):
    """Q symmetric FP64 with integer entries, b FP64 (zeros unless b_range)."""
    g = rng_for(_TAG_RANDOM, n, seed)
    mask = g.random((n, n)) < density
    vals = g.integers(lo, hi + 1, size=(n, n)).astype(np.float64)
    Q = _mirror_upper(np.where(mask, vals, 0.0))
    if b_range is None:
        b = np.zeros(n)
    else:
        b = g.integers(b_range[0], b_range[1] + 1, size=n).astype(np.float64)
    return np.ascontiguousarray(Q), b


def dense_ubqp(n: int, seed: int, lo: int = -100, hi: int = 100, b_lo: int = -50, b_hi: int = 50):
    """Fully dense integer instance with integer linear term."""
    g = rng_for(_TAG_DENSE, n, seed)
    Q = _mirror_upper(g.integers(lo, hi + 1, size=(n, n)).astype(np.float64))
    b = g.integers(b_lo, b_hi + 1, size=n).astype(np.float64)
    return np.ascontiguousarray(Q), b


def maxcut_ubqp(n: int, density: float, seed: int):
    """Max-Cut on G(n, density) with +-1 weights as a 0/1 UBQP with f = -cut."""
    g = rng_for(_TAG_MAXCUT, n, seed)
    mask = g.random((n, n)) < density
    sgn = np.where(g.random((n, n)) < 0.5, -1.0, 1.0)
    U = np.triu(np.where(mask, sgn, 0.0), 1)
    W = U + U.T
    return np.ascontiguousarray(W), -W.sum(axis=1)


def perturbation(Q: np.ndarray, seed: int, sigma_rel: float = 1e-3) -> np.ndarray:
    """Symmetric mu with mu_ij ~ N(0, sigma) on the stored (nonzero or diagonal)
    entries of Q, sigma = sigma_rel * max |Q_ij| over the off-diagonal (or 1 when
    the off-diagonal is empty).  Zero off-diagonal entries stay zero."""
    n = Q.shape[0]
    off = np.abs(Q - np.diag(np.diag(Q)))
    scale = float(off.max()) if n > 1 and off.max() > 0 else 1.0
    sigma = sigma_rel * scale
    g = rng_for(_TAG_MU, n, seed)
    z = g.standard_normal((n, n)) * sigma
    keep = (Q != 0) | np.eye(n, dtype=bool)
    return np.ascontiguousarray(_mirror_upper(np.where(keep, z, 0.0)))


def random_starts(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` starting points uniform in [0,1]^n, shape (count, n)."""
    return rng_for(_TAG_STARTS, n, seed).random((count, n))


def box_points(n: int, count: int, seed: int) -> np.ndarray:
    """Points uniform in the box, shape (count, n)."""
    return rng_for(_TAG_BOX, n, seed).random((count, n))


# ---- the five workload families ---------------------------------------------------

def c1_instance(n: int = 50, seed: int = 0):
    """Single-instance case: density 0.1, integers in [-100, 100], b = 0."""
    return random_ubqp(n, 0.1, seed)


def c2_instance(n: int, seed: int):
    """Sweep case: n in {250, 500, 1000, 2500}, same law as c1."""
    return random_ubqp(n, 0.1, seed)


def c3_instance(n: int = 1000, seed: int = 1):
    """Differentiable-objective case: dense Q in [-100,100], b in [-50,50]."""
    return dense_ubqp(n, seed)


def c4_instance(n: int = 2500, seed: int = 2):
    """Restart-batch case: density 0.1 as c2 (one instance shared by all starts)."""
    return random_ubqp(n, 0.1, seed)


def c5_specs(count: int = 512, seed: int = 3, n_lo: int = 100, n_hi: int = 3000):
    """Sizes, densities and kinds of the ragged batch: list of (n, density, kind, seed)."""
    g = rng_for(_TAG_C5, count, seed)
    ns = g.integers(n_lo, n_hi + 1, size=count)
    dens = g.uniform(0.05, 1.0, size=count)
    kinds = np.array(["int" if i % 2 == 0 else "maxcut" for i in range(count)])
    return [(int(ns[i]), float(dens[i]), str(kinds[i]), seed * 100003 + i) for i in range(count)]


def c5_instance(spec):
    """One instance of the ragged batch from a ``c5_specs`` entry."""
    n, dens, kind, s = spec
    if kind == "int":
        return random_ubqp(n, dens, s)
    return maxcut_ubqp(n, dens, s)
