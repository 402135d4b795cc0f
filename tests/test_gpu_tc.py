"""GPU checks of the tensor-core contraction (tcgen05 + TMA + TMEM, split-K over a
cluster) through the C ABI, against the exact product of the same BF16 operands.

Q_off entries are integers in [-100, 100] (exact in BF16); the iterate is split into two
BF16 terms x = hi + lo.  FP32 accumulation of n products: the bar is 1e-6 relative to
sum_k |A_ik| |B_rk| (rounding of the accumulation order only)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bf16_bits(a):
    import torch
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16).copy(), t.float().numpy().astype(np.float64)


def _probe(A, Bhi, Blo, cluster=0):
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    L.ubqp_tc_matmul_probe.restype = C.c_int
    n, R = A.shape[0], Bhi.shape[0]
    D = np.zeros((R, n), np.float32)
    rc = L.ubqp_tc_matmul_probe(A.ctypes.data_as(C.c_void_p), Bhi.ctypes.data_as(C.c_void_p),
                                None if Blo is None else Blo.ctypes.data_as(C.c_void_p), C.c_int64(n), C.c_int64(R),
                                C.c_int32(cluster), D.ctypes.data_as(C.c_void_p))
    assert rc == 0, rc
    return D


@pytest.mark.parametrize("n,R,cluster,two", [
    (128, 16, 1, True), (200, 37, 0, True), (1000, 64, 2, True), (1000, 256, 0, True),
    (2500, 256, 0, True), (640, 300, 0, True), (384, 48, 3, False), (2560, 256, 4, True)])
def test_tc_contraction_matches_exact_product(n, R, cluster, two):
    rng = np.random.default_rng(n + R)
    A = rng.integers(-100, 101, (n, n)).astype(np.float32)
    A = np.triu(A) + np.triu(A, 1).T
    np.fill_diagonal(A, 0)
    X = rng.random((R, n))
    Ab, Af = _bf16_bits(A)
    hb, hf = _bf16_bits(X)
    lb, lf = _bf16_bits(X - hf) if two else (None, 0.0)
    D = _probe(Ab, hb, lb, cluster).astype(np.float64)
    B = hf + (lf if two else 0.0)
    ref = B @ Af.T                       # exact in FP64 for these operands
    scale = np.abs(B) @ np.abs(Af).T
    err = np.max(np.abs(D - ref) / np.maximum(scale, 1.0))
    assert err <= 1e-6, err
    if two:   # the two-term split represents x to about 2^-16
        assert np.max(np.abs(B - X)) <= 2 ** -15
