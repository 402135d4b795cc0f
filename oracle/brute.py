"""Exhaustive minimum of f(x) = x^T Q x + b^T x over {0,1}^n (Eq. (bqp)).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The plain definition of the
optimum: every one of the 2^n points is evaluated, in chunks, with numpy in FP64.
Usable up to n of about 22.
"""
from __future__ import annotations

import numpy as np


def enumerate_min(Q, b=None, chunk_bits: int = 15):
    """Return (f*, x*) with x* the first minimiser in counting order."""
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[0]
    b = np.zeros(n) if b is None else np.asarray(b, dtype=np.float64)
    best, arg = np.inf, 0
    step = 1 << min(chunk_bits, n)
    bits = np.arange(n)
    for start in range(0, 1 << n, step):
        idx = np.arange(start, start + step, dtype=np.int64)
        X = ((idx[:, None] >> bits) & 1).astype(np.float64)
        F = np.einsum("ij,jk,ik->i", X, Q, X) + X @ b
        k = int(np.argmin(F))
        if F[k] < best:
            best, arg = float(F[k]), int(idx[k])
    x = ((arg >> bits) & 1).astype(np.uint8)
    return best, x
