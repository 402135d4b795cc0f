"""ubqp_penalized_eval_noalloc against ubqp_penalized_eval, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc (they manage all
device memory themselves, or cannot afford the device-wide synchronization it may cause); it
keeps its scratch in a static device array that every call reuses.  Calls in a row, each
compared with the allocating entry point on the same inputs, check that the reused scratch
carries nothing from one call into the next, including a small call after a large one.
This file is collected last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2408_04875_gb300 import instances as I

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-5, "float64": 1e-12}    # the tolerances of the penalized-objective tests


def _lib():
    import paper_2408_04875_gb300 as ub
    return ub.lib()


def _call(fn, Q, b, p, X, torch):
    code = 1 if X.dtype == torch.float64 else 0
    h = torch.empty(X.shape[0], dtype=X.dtype, device=X.device)
    g = torch.empty_like(X)
    s = torch.cuda.current_stream().cuda_stream
    rc = fn(Q.data_ptr(), None if b is None else b.data_ptr(), None if p is None else p.data_ptr(), X.data_ptr(),
            Q.shape[0], X.shape[0], code, h.data_ptr(), g.data_ptr(), s)
    assert rc == 0, _lib().ubqp_last_error()
    return h.double().cpu().numpy(), g.double().cpu().numpy()


def _compare(Q, b, p, X, torch, what):
    L = _lib()
    h_ref, g_ref = _call(L.ubqp_penalized_eval, Q, b, p, X, torch)
    h_new, g_new = _call(L.ubqp_penalized_eval_noalloc, Q, b, p, X, torch)
    tol = TOL[str(X.dtype).replace("torch.", "")]
    assert np.max(np.abs(g_new - g_ref)) <= tol * max(np.max(np.abs(g_ref)), 1.0), what
    assert np.max(np.abs(h_new - h_ref) / np.maximum(np.abs(h_ref), 1.0)) <= tol, what


def _data(n, batch, dt, seed, torch):
    rng = np.random.default_rng(seed)
    Q = rng.integers(-100, 101, (n, n)).astype(np.float64)
    Q = np.triu(Q) + np.triu(Q, 1).T
    b = rng.integers(-50, 51, n).astype(np.float64)
    p = rng.uniform(0, 100, n)
    X = rng.random((batch, n))
    return tuple(torch.tensor(a, dtype=dt, device="cuda") for a in (Q, b, p, X))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_noalloc_matches_allocating_entry_point_twice(dtype):
    """The C3 matrix (n = 1000, dense) with 64 points, two calls in a row on different points."""
    import torch
    dt = getattr(torch, dtype)
    Q, b = I.c3_instance(1000, 1)
    p = np.random.default_rng(1).uniform(0, 100, 1000)
    Qt, bt, pt = (torch.tensor(a, dtype=dt, device="cuda") for a in (Q, b, p))
    for call, seed in enumerate((1, 2)):
        X = torch.tensor(I.box_points(1000, 64, seed), dtype=dt, device="cuda")
        _compare(Qt, bt, pt, X, torch, f"call {call}")


def test_noalloc_shapes_in_a_row_large_then_small():
    """A sequence on the shared scratch: the largest work partition (n = 2500, 256 points: 256
    rows per item), then a smaller one (n = 1000, 64 points), then a small ragged one
    (n = 300, 5 points, b and p absent), then the first again."""
    import torch
    seq = [(2500, 256, 3), (1000, 64, 4), (300, 5, 5), (2500, 256, 3)]
    for n, batch, seed in seq:
        Q, b, p, X = _data(n, batch, torch.float32, seed, torch)
        if n == 300:
            b = p = None
        _compare(Q, b, p, X, torch, (n, batch))


def test_noalloc_fp64_near_the_size_limit():
    """FP64 with n = 25600 (one point is 200 KiB, the limit)."""
    import torch
    n = 25600
    g = torch.Generator(device="cuda").manual_seed(0)
    Q = torch.randint(-100, 101, (n, n), device="cuda", generator=g).double()
    Q = torch.triu(Q) + torch.triu(Q, 1).T
    b = torch.randint(-50, 51, (n,), device="cuda", generator=g).double()
    X = torch.rand((2, n), device="cuda", generator=g, dtype=torch.float64)
    _compare(Q, b, None, X, torch, "n=25600")
    del Q


@pytest.mark.parametrize("case,msg", [("batch", b"256 points"), ("n", b"200 KiB"), ("items", b"work items")])
def test_noalloc_rejects_sizes_beyond_its_scratch(case, msg):
    import torch
    L = _lib()
    n, batch, dt = {"batch": (8, 300, torch.float32), "n": (51201, 1, torch.float32),
                    "items": (20000, 256, torch.float32)}[case]
    Q = torch.zeros((1, 1), dtype=dt, device="cuda")     # the sizes are checked before any access
    X = torch.zeros((1, 1), dtype=dt, device="cuda")
    rc = L.ubqp_penalized_eval_noalloc(Q.data_ptr(), None, None, X.data_ptr(), n, batch, 0, None, None, None)
    assert rc == -1
    assert msg in L.ubqp_last_error(), L.ubqp_last_error()
