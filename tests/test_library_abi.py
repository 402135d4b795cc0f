"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, exports
every function include/ubqp.h declares, and its option/stat structs have the layout
the header gives (no compute calls: there is no GPU here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "ubqp.h")


@pytest.fixture(scope="module")
def built():
    from paper_2408_04875_gb300 import build_lib
    return build_lib.build()


def _declared_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ubqp_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = _declared_functions()
    for want in ("ubqp_solve", "ubqp_solve_batched", "ubqp_penalized_eval", "ubqp_inner_run",
                 "ubqp_opts_default", "ubqp_status_string", "ubqp_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ubqp_[a-z0-9_]+)", out))
    missing = [f for f in _declared_functions() if f not in exported]
    assert not missing, missing


def test_struct_layout_matches_header(built, tmp_path):
    src = tmp_path / "s.c"
    src.write_text('#include <stdio.h>\n#include "ubqp.h"\n#include <stddef.h>\n'
                   'int main(){printf("%zu %zu %zu %zu\\n", sizeof(ubqp_opts), sizeof(ubqp_stats),'
                   ' offsetof(ubqp_opts, stream), offsetof(ubqp_stats, inner_hist));return 0;}\n')
    exe = tmp_path / "s"
    subprocess.run(["gcc", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    import paper_2408_04875_gb300 as ub
    assert vals == [C.sizeof(ub.Opts), C.sizeof(ub.Stats), ub.Opts.stream.offset, ub.Stats.inner_hist.offset]


def test_defaults_and_status_strings(built):
    import paper_2408_04875_gb300 as ub
    o = ub.opts()
    assert (o.max_outer, o.max_inner, o.tol_inner, o.eta) == (1000, 10000, 1e-5, 0.9)
    L = ub.lib()
    assert L.ubqp_status_string(-2) == b"UBQP_ENOTSYM"
    assert L.ubqp_status_string(1) == b"UBQP_EMAXITER"


def test_argument_errors_need_no_gpu(built):
    """Invalid sizes are rejected before any CUDA call."""
    import numpy as np
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    n = np.array([0], np.int64)
    q = np.zeros(1)
    ptrs = (C.c_void_p * 1)(q.ctypes.data)
    x = np.zeros(1, np.uint8)
    xp = (C.c_void_p * 1)(x.ctypes.data)
    obj = np.zeros(1)
    rc = L.ubqp_solve_batched(1, n.ctypes.data, C.cast(ptrs, C.c_void_p), None, None,
                              C.cast(xp, C.c_void_p), obj.ctypes.data)
    assert rc == -1
    assert b"out of" in L.ubqp_last_error()


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2408_04875_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "ubqp_oracle" not in txt, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every entry point raises before computing anything: there
    is no CPU fallback in the product path."""
    import numpy as np
    import paper_2408_04875_gb300 as ub
    monkeypatch.setattr(ub, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(ub, "_lib", None)
    Q = np.eye(4)
    x = np.full(4, 0.5)
    calls = [lambda: ub.solve(Q), lambda: ub.solve_batched([Q]), lambda: ub.initial_point(Q),
             lambda: ub.inner_run(Q, np.zeros(4), 1.0, x), lambda: ub.penalty_probe(Q, np.zeros(4), 1.0, x),
             lambda: ub.opts()]
    for call in calls:
        with pytest.raises(RuntimeError, match="missing"):
            call()


@pytest.mark.parametrize("kw,msg", [
    (dict(method=7), "method"), (dict(max_outer=-1), "max_outer"), (dict(max_inner=-1), "max_inner"),
    (dict(eta=0.0), "eta"), (dict(eta=1.0), "eta"), (dict(eta=float("nan")), "eta"),
    (dict(tol_inner=0.0), "tolerances"), (dict(tol_outer=-1.0), "tolerances"),
    (dict(alpha_min=0.0), "clamp"), (dict(alpha_min=2.0, alpha_max=1.0), "clamp"),
    (dict(restarts=-1), "restarts"), (dict(restarts=4097), "restarts"),
    (dict(precision=9), "precision"), (dict(lobpcg_max_iter=0), "iteration caps"),
    (dict(jacobi_max_iter=0), "iteration caps"), (dict(max_ticks_per_sync=0), "max_ticks_per_sync"),
    (dict(max_ticks_per_sync=4097), "max_ticks_per_sync"), (dict(sigma_rel=-1.0), "sigma_rel"),
    (dict(gamma_margin=0.0), "gamma_margin"), (dict(tc_cluster=9), "tc_cluster"),
    (dict(gemv_kernel=4), "gemv_kernel"), (dict(lane_budget=-1), "lane_budget"),
    (dict(rows_per_item=12), "rows_per_item"), (dict(rows_per_item=4), "rows_per_item"),
    (dict(rows_per_item=264), "rows_per_item"), (dict(wait_limit_us=-1), "wait_limit_us"),
    (dict(tc_fuse=2), "tc_fuse"), (dict(sparse_storage=3), "sparse_storage"),
])
def test_invalid_options_are_rejected_before_any_cuda_call(built, kw, msg):
    """Every option outside its documented range returns UBQP_EINVAL with a message naming
    it, before the library touches the device (so this runs without a GPU)."""
    import numpy as np
    import paper_2408_04875_gb300 as ub
    with pytest.raises(ub.UBQPError) as e:
        ub.solve(np.eye(3), **kw)
    assert e.value.status == -1 and msg in str(e.value)


def test_restart_tuner_with_caller_starts_is_rejected_without_gpu(built):
    import numpy as np
    import paper_2408_04875_gb300 as ub
    with pytest.raises(ub.UBQPError) as e:
        ub.solve(np.eye(3), starts=np.full((2, 3), 0.5), restarts=0)
    assert e.value.status == -1 and "tuner" in str(e.value)


def _solve_batched_raw(L, num, ns, q_null=False, x_null=False, obj_null=False):
    import numpy as np
    n = np.array(ns if ns else [1], np.int64)
    qs = [np.zeros(max(k, 1) ** 2) for k in n]
    xs = [np.zeros(max(k, 1), np.uint8) for k in n]
    qp = (C.c_void_p * len(n))(*[None if q_null else q.ctypes.data for q in qs])
    xp = (C.c_void_p * len(n))(*[x.ctypes.data for x in xs])
    obj = np.zeros(len(n))
    return L.ubqp_solve_batched(num, n.ctypes.data, C.cast(qp, C.c_void_p), None, None,
                                None if x_null else C.cast(xp, C.c_void_p), None if obj_null else obj.ctypes.data)


@pytest.mark.parametrize("case,msg", [
    (dict(num=0, ns=[]), b"num >= 1"),
    (dict(num=1, ns=[65537]), b"n = 65537 out of [1, 65536]"),
    (dict(num=1, ns=[-3]), b"n = -3 out of"),
    (dict(num=2, ns=[4, 0]), b"instance 1: n = 0 out of"),
    (dict(num=1, ns=[4], q_null=True), b"null Q or x_out"),
    (dict(num=1, ns=[4], x_null=True), b"non-null n, Q, x_out, obj_out"),
    (dict(num=1, ns=[4], obj_null=True), b"non-null n, Q, x_out, obj_out"),
])
def test_sizes_and_null_pointers_rejected_without_gpu(built, case, msg):
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    assert _solve_batched_raw(L, **case) == -1
    assert msg in L.ubqp_last_error()


def test_last_error_is_per_thread(built):
    """ubqp_last_error is thread-local: an error on one thread is not seen on another."""
    import threading
    import numpy as np
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    seen = {}

    def fail():
        try:
            ub.solve(np.eye(3), eta=2.0)
        except ub.UBQPError:
            pass
        seen["a"] = L.ubqp_last_error()

    def fresh():
        seen["b"] = L.ubqp_last_error()

    ta = threading.Thread(target=fail)
    ta.start()
    ta.join()
    tb = threading.Thread(target=fresh)
    tb.start()
    tb.join()
    assert b"eta" in seen["a"] and seen["b"] == b""
