"""Python binding of libubqp.so, the GB300 implementation of the vectorized PSDP
method for unconstrained binary quadratic programs (arXiv 2408.04875).

Argument marshalling only: every step of the method runs in the CUDA library.  The
library is built in-tree by ``paper_2408_04875_gb300.build_lib.build()`` (or
``__graft_entry__.build()``); calling any solver function without it raises.

Arrays may be numpy arrays (host memory) or torch tensors (CUDA tensors are passed to
the library as device pointers; CPU tensors go through numpy).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = ["lib", "Opts", "Stats", "opts", "solve", "solve_batched", "penalized_eval", "penalized_vjp", "inner_run",
           "penalty_probe", "initial_point", "PenalizedObjective", "UBQPError", "PABB", "PPA", "FP32",
           "BF16X2_TC", "BF16_TC", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libubqp.so")
PABB, PPA = 0, 1
FP32, BF16X2_TC, BF16_TC = 0, 1, 2
HIST_BINS = 101
_lock = threading.Lock()
_lib = None


class UBQPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Stats(C.Structure):
    _fields_ = [("inner_iters", C.c_int64), ("inner_steps", C.c_int64), ("var_updates", C.c_int64),
                ("outer_steps", C.c_int64), ("lobpcg_iters", C.c_int64), ("jacobi_iters", C.c_int64),
                ("floor_steps", C.c_int64), ("ticks", C.c_int64), ("lanes", C.c_int64),
                ("lanes_capped", C.c_int64), ("ms_device", C.c_double), ("ms_total", C.c_double),
                ("phase_a_ms", C.c_double), ("phase_a_launches", C.c_int64), ("phase_a_bytes", C.c_int64),
                ("kernel_launches", C.c_int64), ("ms_to_target", C.c_double), ("phase_a_flops", C.c_int64),
                ("cluster_size", C.c_int32), ("gemv_kernel", C.c_int32), ("restarts", C.c_int32),
                ("restart_probe_us", C.c_float * 5), ("tc_kernel", C.c_int32), ("sym_storage", C.c_int32),
                ("inner_hist", C.c_int64 * HIST_BINS), ("alg_bytes", C.c_int64), ("alg_flops", C.c_int64),
                ("cluster_probe_us", C.c_float * 9), ("cluster_tuned", C.c_int32), ("storage", C.c_int32)]

    def as_dict(self):
        arrays = ("inner_hist", "restart_probe_us", "cluster_probe_us")
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in arrays}
        for k in arrays:
            d[k] = list(getattr(self, k))
        return d


class Opts(C.Structure):
    _fields_ = [("method", C.c_int), ("max_outer", C.c_int), ("max_inner", C.c_int),
                ("tol_inner", C.c_double), ("tol_outer", C.c_double), ("eta", C.c_double),
                ("gamma_margin", C.c_double), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("tau_z", C.c_double), ("eps_hp_rel", C.c_double), ("lambda_floor_rel", C.c_double),
                ("sigma_rel", C.c_double), ("seed", C.c_uint64), ("restarts", C.c_int),
                ("precision", C.c_int), ("lobpcg_max_iter", C.c_int), ("lobpcg_tol", C.c_double),
                ("jacobi_max_iter", C.c_int), ("max_ticks_per_sync", C.c_int), ("profile_kernels", C.c_int),
                ("stop_at_target", C.c_int), ("tc_cluster", C.c_int), ("gemv_kernel", C.c_int), ("lane_budget", C.c_int), ("rows_per_item", C.c_int), ("sym_storage", C.c_int),
                ("wait_limit_us", C.c_int), ("tc_fuse", C.c_int), ("sparse_storage", C.c_int),
                ("target_objective", C.c_double),
                ("stream", C.c_void_p),
                ("mu", C.c_void_p), ("x_starts", C.c_void_p), ("stats", C.POINTER(Stats))]


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = C.CDLL(LIB_PATH)
            vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
            L.ubqp_opts_default.argtypes = [C.POINTER(Opts)]
            L.ubqp_status_string.restype = C.c_char_p
            L.ubqp_status_string.argtypes = [C.c_int]
            L.ubqp_last_error.restype = C.c_char_p
            L.ubqp_solve.argtypes = [vp, vp, i64, C.POINTER(Opts), vp, vp]
            L.ubqp_solve_batched.argtypes = [i32, vp, vp, vp, C.POINTER(Opts), vp, vp]
            L.ubqp_penalized_eval.argtypes = [vp, vp, vp, vp, i64, i64, C.c_int, vp, vp, vp]
            L.ubqp_penalized_vjp.argtypes = [vp, vp, vp, i64, i64, C.c_int, vp, vp, vp, vp]
            L.ubqp_penalized_eval_noalloc.argtypes = [vp, vp, vp, vp, i64, i64, C.c_int, vp, vp, vp]
            L.ubqp_inner_run.argtypes = [vp, vp, vp, vp, i64, C.POINTER(Opts), i32, vp, vp, vp,
                                         C.POINTER(i32), C.POINTER(i32)]
            L.ubqp_penalty_probe.argtypes = [vp, vp, vp, vp, i64, C.POINTER(Opts), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(i32), C.POINTER(i32)]
            L.ubqp_initial_point.argtypes = [vp, vp, vp, i64, C.POINTER(Opts), vp, vp]
            for name in ("ubqp_solve", "ubqp_solve_batched", "ubqp_penalized_eval", "ubqp_penalized_vjp",
                         "ubqp_penalized_eval_noalloc", "ubqp_inner_run", "ubqp_penalty_probe",
                         "ubqp_initial_point"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc < 0:
        L = lib()
        raise UBQPError(rc, f"{what}: {L.ubqp_status_string(rc).decode()}: {L.ubqp_last_error().decode()}")
    return rc


def opts(**kw) -> Opts:
    o = Opts()
    lib().ubqp_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


# --- array marshalling -----------------------------------------------------------------

def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _as_f64(a, keep):
    """Pointer to FP64 data: CUDA tensors stay on the device, everything else becomes a
    contiguous host array (kept alive in ``keep``)."""
    if a is None:
        return None
    if _is_cuda_tensor(a):
        import torch
        t = a.detach().to(torch.float64).contiguous()
        keep.append(t)
        return t.data_ptr()
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    arr = np.ascontiguousarray(a, dtype=np.float64)
    keep.append(arr)
    return arr.ctypes.data


def _ptr_array(ptrs, keep):
    arr = (C.c_void_p * len(ptrs))(*[p if p is not None else 0 for p in ptrs])
    keep.append(arr)
    return C.cast(arr, C.c_void_p)


# --- solver entry points ------------------------------------------------------------------

def solve_batched(Qs, bs=None, mus=None, starts=None, **kw):
    """Alg. 3 on a list of instances.  Returns (list of uint8 x, float64 objectives, stats).
    ``mus``: optional per-instance perturbations; ``starts``: optional per-instance
    (restarts-1) x n extra starting points."""
    keep = []
    num = len(Qs)
    n = np.array([np.shape(Q)[0] for Q in Qs], dtype=np.int64)
    keep.append(n)
    qp = [_as_f64(Q, keep) for Q in Qs]
    bp = [_as_f64(b, keep) for b in bs] if bs is not None else [None] * num
    o = opts(**kw)
    if mus is not None:
        o.mu = _ptr_array([_as_f64(m, keep) for m in mus], keep).value
    if starts is not None:
        o.x_starts = _ptr_array([_as_f64(s, keep) for s in starts], keep).value
    st = Stats()
    o.stats = C.pointer(st)
    xs = [np.zeros(int(k), np.uint8) for k in n]
    xp = [x.ctypes.data for x in xs]
    obj = np.zeros(num, np.float64)
    rc = lib().ubqp_solve_batched(num, n.ctypes.data, _ptr_array(qp, keep), _ptr_array(bp, keep), C.byref(o),
                                  _ptr_array(xp, keep), obj.ctypes.data)
    _check(rc, "ubqp_solve_batched")
    d = st.as_dict()
    d["status"] = rc
    return xs, obj, d


def solve(Q, b=None, mu=None, starts=None, **kw):
    """Alg. 3 on one instance.  Returns (uint8 x, objective, stats)."""
    xs, obj, st = solve_batched([Q], None if b is None else [b], None if mu is None else [mu],
                                None if starts is None else [starts], **kw)
    return xs[0], float(obj[0]), st


def inner_run(Qp, bp, p, x0, trace_len: int = 0, **kw):
    """Test entry: Alg. 2 (or Alg. 1) from a given state on the FP32 GPU path."""
    keep = []
    n = int(np.shape(Qp)[0])
    o = opts(**kw)
    tx = np.zeros((max(trace_len, 1), n)) if trace_len else None
    ta = np.zeros(max(trace_len, 1)) if trace_len else None
    xo = np.zeros(n)
    steps, code = C.c_int32(0), C.c_int32(0)
    rc = lib().ubqp_inner_run(_as_f64(Qp, keep), _as_f64(bp, keep), _as_f64(p, keep), _as_f64(x0, keep), n,
                              C.byref(o), trace_len, None if tx is None else tx.ctypes.data,
                              None if ta is None else ta.ctypes.data, xo.ctypes.data, C.byref(steps),
                              C.byref(code))
    _check(rc, "ubqp_inner_run")
    return {"x": xo, "steps": steps.value, "exit": code.value, "trace_x": tx, "trace_alpha": ta}


def penalty_probe(Qp, bp, p, x, **kw):
    """Test entry: one penalty step (lambda_min, alpha) on the GPU."""
    keep = []
    n = int(np.shape(Qp)[0])
    o = opts(**kw)
    lam, alpha = C.c_double(0), C.c_double(0)
    m, it = C.c_int32(0), C.c_int32(0)
    rc = lib().ubqp_penalty_probe(_as_f64(Qp, keep), _as_f64(bp, keep), _as_f64(p, keep), _as_f64(x, keep), n,
                                  C.byref(o), C.byref(lam), C.byref(alpha), C.byref(m), C.byref(it))
    _check(rc, "ubqp_penalty_probe")
    return {"lambda": lam.value, "alpha": alpha.value, "n_active": m.value, "iters": it.value}


def initial_point(Q, b=None, mu=None, **kw):
    """Test entry: device initialization of Sec. 3.5; returns (x0, gamma)."""
    keep = []
    n = int(np.shape(Q)[0])
    o = opts(**kw)
    x0, gam = np.zeros(n), np.zeros(n)
    rc = lib().ubqp_initial_point(_as_f64(Q, keep), _as_f64(b, keep), _as_f64(mu, keep), n, C.byref(o),
                                  x0.ctypes.data, gam.ctypes.data)
    _check(rc, "ubqp_initial_point")
    return x0, gam


def penalized_eval(Q, b, p, x, want_h: bool = True, want_g: bool = True, stream=None):
    """h(x,p) and grad h for CUDA tensors Q (n,n), b/p (n) or None, x (batch,n) or (n,)."""
    import torch
    if not (_is_cuda_tensor(Q) and _is_cuda_tensor(x)):
        raise ValueError("penalized_eval takes CUDA tensors")
    dt = Q.dtype
    if dt not in (torch.float32, torch.float64):
        raise ValueError("float32 or float64 tensors required")
    code = 1 if dt == torch.float64 else 0
    squeeze = x.dim() == 1
    X = x.reshape(1, -1) if squeeze else x
    n = Q.shape[0]
    Qc = Q.contiguous()
    Xc = X.to(dt).contiguous()
    bc = None if b is None else b.to(dt).contiguous()
    pc = None if p is None else p.to(dt).contiguous()
    h = torch.empty(Xc.shape[0], dtype=dt, device=Q.device) if want_h else None
    g = torch.empty_like(Xc) if want_g else None
    s = stream if stream is not None else torch.cuda.current_stream(Q.device).cuda_stream
    rc = lib().ubqp_penalized_eval(Qc.data_ptr(), None if bc is None else bc.data_ptr(),
                                   None if pc is None else pc.data_ptr(), Xc.data_ptr(), n, Xc.shape[0], code,
                                   None if h is None else h.data_ptr(), None if g is None else g.data_ptr(), s)
    _check(rc, "ubqp_penalized_eval")
    if squeeze:
        h = None if h is None else h[0]
        g = None if g is None else g[0]
    return h, g


def penalized_vjp(x, g, grad_h, want_x=True, want_p=False, want_b=False, stream=None):
    """Backward of penalized_eval for CUDA tensors x, g (batch, n) or (n,) and grad_h (batch,)
    or a scalar: returns (grad_h * g, sum_r grad_h[r] (x_r - x_r^2), sum_r grad_h[r] x_r), each
    None unless asked for."""
    import torch
    squeeze = x.dim() == 1
    X = x.reshape(1, -1) if squeeze else x
    dt = X.dtype
    code = 1 if dt == torch.float64 else 0
    Xc = X.contiguous()
    Gc = g.reshape(Xc.shape).to(dt).contiguous()
    go = grad_h.reshape(-1).to(dt).contiguous()
    gx = torch.empty_like(Xc) if want_x else None
    gp = torch.empty(Xc.shape[1], dtype=dt, device=Xc.device) if want_p else None
    gb = torch.empty(Xc.shape[1], dtype=dt, device=Xc.device) if want_b else None
    s = stream if stream is not None else torch.cuda.current_stream(Xc.device).cuda_stream
    rc = lib().ubqp_penalized_vjp(Xc.data_ptr(), Gc.data_ptr(), go.data_ptr(), Xc.shape[1], Xc.shape[0], code,
                                  None if gx is None else gx.data_ptr(), None if gp is None else gp.data_ptr(),
                                  None if gb is None else gb.data_ptr(), s)
    _check(rc, "ubqp_penalized_vjp")
    if squeeze and gx is not None:
        gx = gx[0]
    return gx, gp, gb


def _make_autograd():
    import torch

    class PenalizedObjective(torch.autograd.Function):
        """h(x, p) = x^T Q x + b^T x + sum_i p_i (x_i - x_i^2) (Sec. 4.1, problem (p)).
        Forward runs ubqp_penalized_eval (the inner loop's GEMV kernel with the gradient
        epilogue) and keeps g; backward runs ubqp_penalized_vjp: grad_out * g for x,
        sum grad_out * (x - x^2) for p and sum grad_out * x for b.  Q is data (no gradient)."""

        @staticmethod
        def forward(ctx, x, Q, b, p):
            h, g = penalized_eval(Q, b, p, x)
            ctx.save_for_backward(x, g)
            ctx.has_b = b is not None
            ctx.has_p = p is not None
            return h

        @staticmethod
        def backward(ctx, grad_out):
            x, g = ctx.saved_tensors
            want_b = ctx.has_b and ctx.needs_input_grad[2]
            want_p = ctx.has_p and ctx.needs_input_grad[3]
            gx, gp, gb = penalized_vjp(x.detach(), g, grad_out.detach(), want_x=ctx.needs_input_grad[0],
                                       want_p=want_p, want_b=want_b)
            return gx, None, gb, gp

    return PenalizedObjective


class _LazyAutograd:
    _cls = None

    def __call__(self):
        if self._cls is None:
            self._cls = _make_autograd()
        return self._cls

    def apply(self, *args):
        return self().apply(*args)


PenalizedObjective = _LazyAutograd()
