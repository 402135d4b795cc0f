"""ctypes wrapper of the FP64 CPU oracle (oracle/ubqp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``.  The CUDA library never imports this module.

``build()`` compiles the oracle with gcc into ``oracle/liboracle.so``; ``lib()``
builds on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "ubqp_oracle.c")]
_HDR = os.path.join(_HERE, "ubqp_oracle.h")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


class Opts(C.Structure):
    _fields_ = [
        ("method", C.c_int), ("max_outer", C.c_int), ("max_inner", C.c_int),
        ("tol_inner", C.c_double), ("tol_outer", C.c_double), ("eta", C.c_double),
        ("gamma_margin", C.c_double), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
        ("tau_z", C.c_double), ("eps_hp_rel", C.c_double), ("lambda_floor_rel", C.c_double),
        ("fp32_noise", C.c_double), ("noise_seed", C.c_ulonglong),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("outer", C.c_int), ("inner_total", C.c_longlong), ("grad_evals", C.c_longlong),
        ("best_outer", C.c_int), ("n_fallback", C.c_int), ("status", C.c_int),
        ("final_binarity", C.c_double),
    ]


def _stale() -> bool:
    if not os.path.exists(_SO):
        return True
    t = os.path.getmtime(_SO)
    return any(os.path.getmtime(p) > t for p in _SRC + [_HDR])


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C11, -O2, no BLAS)."""
    with _lock:
        if force or _stale():
            tmp = _SO + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path: str):
    """Open a compiled oracle at ``path`` and declare its entry points (the tests also
    load copies of the oracle with planted mistakes this way)."""
    L = C.CDLL(path)
    L.orc_opts_default.argtypes = [C.POINTER(Opts)]
    L.orc_objective.restype = C.c_double
    L.orc_objective.argtypes = [C.c_int, _dp, C.c_void_p, _u8]
    L.orc_reformulate.argtypes = [C.c_int, _dp, C.c_void_p, C.c_void_p, C.c_double, _dp, _dp, _dp]
    L.orc_initial_point.restype = C.c_int
    L.orc_initial_point.argtypes = [C.c_int, _dp, _dp, _dp]
    L.orc_penalized.restype = C.c_double
    L.orc_penalized.argtypes = [C.c_int, _dp, C.c_void_p, C.c_void_p, _dp, C.c_void_p]
    L.orc_kkt_residual.restype = C.c_double
    L.orc_kkt_residual.argtypes = [C.c_int, _dp, _dp]
    L.orc_rho.restype = C.c_double
    L.orc_rho.argtypes = [C.c_int, _dp, C.c_void_p, C.c_void_p]
    L.orc_lambda_min.restype = C.c_double
    L.orc_lambda_min.argtypes = [C.c_int, _dp]
    L.orc_penalty_step.restype = C.c_double
    L.orc_penalty_step.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.POINTER(Opts), C.c_int,
                                   C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.orc_inner.restype = C.c_int
    L.orc_inner.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.POINTER(Opts), C.c_int,
                            C.c_void_p, C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
    L.orc_solve.restype = C.c_int
    L.orc_solve.argtypes = [C.c_int, _dp, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Opts),
                            _u8, C.POINTER(C.c_double), C.POINTER(Stats), C.c_void_p, _dp]
    return L


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def opts(**kw) -> Opts:
    o = Opts()
    lib().orc_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def objective(Q, b, x) -> float:
    Q = _c(Q)
    n = Q.shape[0]
    b = None if b is None else _c(b)
    return lib().orc_objective(n, Q, _ptr(b), _c(x, np.uint8))


def reformulate(Q, b=None, mu=None, margin: float = 1.0):
    Q = _c(Q)
    n = Q.shape[0]
    b = None if b is None else _c(b)
    mu = None if mu is None else _c(mu)
    Qp = np.empty_like(Q)
    bp = np.empty(n)
    gam = np.empty(n)
    lib().orc_reformulate(n, Q, _ptr(b), _ptr(mu), margin, Qp, bp, gam)
    return Qp, bp, gam


def initial_point(Qp, bp):
    Qp = _c(Qp)
    x = np.empty(Qp.shape[0])
    rc = lib().orc_initial_point(Qp.shape[0], Qp, _c(bp), x)
    if rc != 0:
        raise ValueError("Q' is not positive definite")
    return x


def penalized(Q, b, p, x, want_grad: bool = True):
    Q = _c(Q)
    n = Q.shape[0]
    b = None if b is None else _c(b)
    p = None if p is None else _c(p)
    g = np.empty(n) if want_grad else None
    h = lib().orc_penalized(n, Q, _ptr(b), _ptr(p), _c(x), _ptr(g))
    return (h, g) if want_grad else h


def kkt_residual(x, g) -> float:
    x = _c(x)
    return lib().orc_kkt_residual(x.shape[0], x, _c(g))


def rho(Q, b=None, p=None) -> float:
    Q = _c(Q)
    b = None if b is None else _c(b)
    p = None if p is None else _c(p)
    return lib().orc_rho(Q.shape[0], Q, _ptr(b), _ptr(p))


def lambda_min(A) -> float:
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    return lib().orc_lambda_min(A.shape[0], A)


def penalty_step(Qp, bp, p, x, o: Opts | None = None, consecutive: int = 0):
    o = o or opts()
    m = C.c_int(0)
    lam = C.c_double(0.0)
    fb = C.c_int(0)
    Qp = _c(Qp)
    a = lib().orc_penalty_step(Qp.shape[0], Qp, _c(bp), _c(p), _c(x), C.byref(o), consecutive,
                               C.byref(m), C.byref(lam), C.byref(fb))
    return a, m.value, lam.value, bool(fb.value)


def inner(Qp, bp, p, x0, o: Opts | None = None, trace_len: int = 0):
    """Run Alg. 2 (or Alg. 1 when o.method == 1) from x0.  Returns a dict with the
    final x, the step count, the exit code and the first ``trace_len`` iterates/steps."""
    o = o or opts()
    Qp = _c(Qp)
    n = Qp.shape[0]
    x = np.array(x0, dtype=np.float64, copy=True)
    tx = np.full((max(trace_len, 1), n), np.nan) if trace_len else None
    ta = np.full(max(trace_len, 1), np.nan) if trace_len else None
    ge = C.c_longlong(0)
    code = C.c_int(0)
    k = lib().orc_inner(n, Qp, _c(bp), _c(p), x, C.byref(o), trace_len, _ptr(tx), _ptr(ta),
                        C.byref(ge), C.byref(code))
    return {"x": x, "steps": k, "grad_evals": ge.value, "exit": code.value,
            "trace_x": tx, "trace_alpha": ta}


def solve(Q, b=None, mu=None, x_start=None, o: Opts | None = None):
    """Alg. 3 in FP64.  Returns (x_best uint8, f_best, stats dict); the stats hold the
    inner step counts (``inner_hist``) and the last penalty vector (``p``)."""
    o = o or opts()
    Q = _c(Q)
    n = Q.shape[0]
    b = None if b is None else _c(b)
    mu = None if mu is None else _c(mu)
    xs = None if x_start is None else _c(x_start)
    xb = np.zeros(n, np.uint8)
    f = C.c_double(0.0)
    st = Stats()
    hist = np.zeros(max(o.max_outer, 1) + 1, np.int32)
    p = np.zeros(n)
    lib().orc_solve(n, Q, _ptr(b), _ptr(mu), _ptr(xs), C.byref(o), xb, C.byref(f), C.byref(st),
                    _ptr(hist), p)
    stats = {k: getattr(st, k) for k, _ in Stats._fields_}
    stats["inner_hist"] = hist[: st.outer].copy()
    stats["p"] = p
    return xb, f.value, stats
