"""ubqp_penalized_eval_noalloc against ubqp_penalized_eval, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc (they manage all
device memory themselves); it keeps its scratch in a static device array that every call
reuses.  Two calls in a row, each compared with the allocating entry point on the same
inputs, check that the reused scratch carries nothing from one call into the next.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2408_04875_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _call(fn, Q, b, p, X, dtype_code, torch):
    h = torch.empty(X.shape[0], dtype=X.dtype, device=X.device)
    g = torch.empty_like(X)
    s = torch.cuda.current_stream().cuda_stream
    rc = fn(C.c_void_p(Q.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(p.data_ptr()), C.c_void_p(X.data_ptr()),
            C.c_int64(Q.shape[0]), C.c_int64(X.shape[0]), C.c_int(dtype_code), C.c_void_p(h.data_ptr()),
            C.c_void_p(g.data_ptr()), C.c_void_p(s))
    assert rc == 0
    return h.double().cpu().numpy(), g.double().cpu().numpy()


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_noalloc_matches_allocating_entry_point_twice(dtype):
    import torch
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    L.ubqp_penalized_eval_noalloc.restype = C.c_int
    dt = getattr(torch, dtype)
    code = 1 if dtype == "float64" else 0
    tol = 1e-5 if dtype == "float32" else 1e-12    # the tolerances of the penalized-objective tests
    Q, b = I.c3_instance(1000, 1)
    p = np.random.default_rng(1).uniform(0, 100, 1000)
    Qt, bt, pt = (torch.tensor(a, dtype=dt, device="cuda") for a in (Q, b, p))
    for call, seed in enumerate((1, 2)):          # two calls in a row on different points
        X = torch.tensor(I.box_points(1000, 64, seed), dtype=dt, device="cuda")
        h_ref, g_ref = _call(L.ubqp_penalized_eval, Qt, bt, pt, X, code, torch)
        h_new, g_new = _call(L.ubqp_penalized_eval_noalloc, Qt, bt, pt, X, code, torch)
        assert np.max(np.abs(g_new - g_ref)) <= tol * np.max(np.abs(g_ref)), f"call {call}"
        assert np.max(np.abs(h_new - h_ref) / np.maximum(np.abs(h_ref), 1.0)) <= tol, f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    Q = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    X = torch.zeros((300, 8), dtype=torch.float32, device="cuda")   # batch > 256
    rc = L.ubqp_penalized_eval_noalloc(C.c_void_p(Q.data_ptr()), None, None, C.c_void_p(X.data_ptr()),
                                       C.c_int64(8), C.c_int64(300), C.c_int(0), None, None, None)
    assert rc == -1
