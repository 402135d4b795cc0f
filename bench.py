"""Benchmark of the vectorized PSDP solver (arXiv 2408.04875) on one node.

A step is one pass of the whole method (initialization, penalty updates with their
lambda_min solves, the PABB inner loops, rounding and exact evaluation) over one batch
of synthetic instances: the plain-PSDP sweep, n in {250, 500, 1000, 2500} x 10 seeded
instances (density 0.1, integers uniform in [-100, 100], b = 0), FP32 path, one start
per instance.  With N ranks (torchrun) every rank solves its own 40 instances (seeds
offset by 10 * rank): weak scaling, no collective on the data path.

Metric: inner projected-gradient iterations x n per second over all lanes (each
gradient evaluation of Alg. 2 on a lane of size n counts n).  Inputs are resident in HBM
when the timed region starts; the FP32 matrices of one batch (302 MB) exceed the 129 MB
L2, so no flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inner PG iters/s (batch×n) and time-to-oracle-objective vs plain FP32 path"
UNIT = "lane-var-updates/s"
GEMV_KERNELS = {1: "phase_a_gemv_kernel", 2: "lane_loop_kernel", 3: "solo_lane_kernel"}
# DRAM bytes (read + write) per algorithmic byte of the dominant kernel, keyed by (scheduler,
# storage), from an ncu capture of every launch of this workload's timed solve
# (dram__bytes_read.sum + dram__bytes_write.sum over the launches against the bench's own
# algorithmic bytes; the C2 launch list under profiles/); other combinations report null
TRAFFIC_RATIO = {(3, 2): 0.7935 / 37.774}
SIZES = (250, 500, 1000, 2500)
SEEDS_PER_SIZE = 10
WORKLOAD = ("plain PSDP sweep: n in {250,500,1000,2500} x 10 seeded instances, density 0.1, "
            "integers in [-100,100], b=0, FP32, 1 start")


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _instances(rank: int, sizes=SIZES, seeds=SEEDS_PER_SIZE):
    from paper_2408_04875_gb300 import instances as I
    Qs, mus = [], []
    for n in sizes:
        for k in range(seeds):
            seed = SEEDS_PER_SIZE * rank + k
            Q, _ = I.c2_instance(n, seed)
            Qs.append(Q)
            mus.append(I.perturbation(Q, seed))
    return Qs, mus


def aggregate_ranks(ms: float, work: float, dist, device: str):
    """Whole-job figures of a multi-rank run: the slowest rank's time (the job ends with it)
    and the work of all ranks.  `dist` is torch.distributed (or None for one rank); the
    tensors live on `device` ("cuda" under NCCL, "cpu" under gloo)."""
    import torch
    ms_t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    work_t = torch.tensor([float(work)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(work_t, op=dist.ReduceOp.SUM)
    return float(ms_t.item()), float(work_t.item())


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks, power, throttle reasons)."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


C4_WORKLOAD = ("batched restarts: n=2500, density 0.1, integers in [-100,100], b=0, 256 starts "
               "(x0 of Eq. (gamma) + 255 uniform), Q_off BF16 on tensor cores with the iterate as two BF16 terms, "
               "FP32 accumulation, diagonal-only perturbation")


def c4_time_to_objective(device: int, restarts: int = 256):
    """The metric's second half, measured once outside the timed sweep: on the batched-restart
    instance (n = 2500, density 0.1, diagonal-only perturbation), the plain FP32 path with one
    start (x^0 of Eq. (gamma)) runs to completion; its objective f32 and device time are the
    reference.  The tensor-core batch (256 starts, BF16 x2 terms) then runs until its best exact
    objective is within 0.1 % of f32 (stop_at_target), and its device time to that point is
    compared.  Clocks are sampled over both runs."""
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    from paper_2408_04875_gb300 import instances as I
    Q, _ = I.c4_instance(2500, 2)
    mu = np.diag(np.diag(I.perturbation(Q, 2)))
    starts = I.random_starts(2500, restarts - 1, 2)
    Qd, Md, Sd = (torch.from_numpy(a).cuda() for a in (Q, mu, starts))
    _, _, swarm = ub.solve(Qd, None, mu=Md, starts=Sd, restarts=restarts, precision=ub.BF16X2_TC,
                           max_outer=1)   # warm-up; its launch-form tuning is cached for the timed call
    sampler = ClockSampler(device)
    sampler.start()
    _, f32, s32 = ub.solve(Qd, None, mu=Md)
    target = f32 + 1e-3 * abs(f32)
    _, ftc, stc = ub.solve(Qd, None, mu=Md, starts=Sd, restarts=restarts, precision=ub.BF16X2_TC,
                           target_objective=target, stop_at_target=1)
    clocks = sampler.stop()
    t_tc = stc["ms_to_target"]
    return {"workload": C4_WORKLOAD, "fp32_single_start": {"objective": f32, "ms": s32["ms_device"],
                                                           "steps": s32["ticks"], "scheduler": s32["gemv_kernel"]},
            "batched": {"restarts": restarts, "best_objective_at_stop": float(ftc), "ms_to_target": t_tc,
                        "steps": stc["ticks"], "tc_kernel": stc["tc_kernel"], "cluster_size": stc["cluster_size"],
                        "us_per_step": (1e3 * t_tc / stc["ticks"]) if stc["ticks"] else None,
                        "contraction_probe_us": {("persistent" if c == 0 else f"split_k_{c}"): t
                                                 for c, t in enumerate(swarm["cluster_probe_us"]) if t > 0}},
            "target": target, "speedup": (s32["ms_device"] / t_tc) if t_tc and t_tc > 0 else None,
            "clocks": clocks}


def run_c4(args):
    """Tensor-core batched path on the batched-restart workload, next to the FP32 path on the
    same instance with one start: throughput, and device time until the batch's best rounded
    objective is within 0.1% of the FP32 single-start result."""
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    from paper_2408_04875_gb300 import instances as I
    torch.cuda.set_device(0)
    Q, b = I.c4_instance(2500, 2)
    mu = np.diag(np.diag(I.perturbation(Q, 2)))
    starts = I.random_starts(2500, args.restarts - 1, 2)
    Qd, Md, Sd = (torch.from_numpy(a).cuda() for a in (Q, mu, starts))
    kw = dict(restarts=args.restarts, precision=ub.BF16X2_TC)
    if args.max_outer is not None:
        kw["max_outer"] = args.max_outer
    _, f32, s32 = ub.solve(Qd, None, mu=Md, **{k: v for k, v in kw.items() if k == "max_outer"})
    target = f32 + 1e-3 * abs(f32)
    for _ in range(args.warmup):
        ub.solve(Qd, None, mu=Md, starts=Sd, target_objective=target, **kw)
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    stats = []
    for _ in range(args.steps):
        _, ftc, st = ub.solve(Qd, None, mu=Md, starts=Sd, target_objective=target,
                              profile_kernels=0 if args.no_profile else 1, **kw)
        stats.append(st)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    work = sum(s["var_updates"] for s in stats)
    pa_ms = sum(s["phase_a_ms"] for s in stats)
    pa_n = sum(s["phase_a_launches"] for s in stats)
    flops = sum(s["phase_a_flops"] for s in stats)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    ach = flops / (pa_ms * 1e-3) / 1e12 if pa_ms > 0 else None
    line = {"metric": METRIC, "value": work / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x2", "data": "synthetic",
            "config": {"workload": C4_WORKLOAD, "restarts": args.restarts, "cluster_size": stats[-1]["cluster_size"],
                       "contraction_probe_us": {("persistent" if c == 0 else f"split_k_{c}"): t
                                                for c, t in enumerate(stats[-1]["cluster_probe_us"]) if t > 0},
                       "fp32_single_start": {"objective": f32, "ms_device": s32["ms_device"]},
                       "batched_best_objective": float(ftc), "ms_to_fp32_objective": stats[-1]["ms_to_target"],
                       "speedup_to_fp32_objective": (s32["ms_device"] / stats[-1]["ms_to_target"]
                                                     if stats[-1]["ms_to_target"] > 0 else None),
                       "ticks_per_step": stats[-1]["ticks"], "l2": "Q_off BF16 13 MB is L2-resident"},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak if ach else None, "traffic": None,
                         "kernel": "phase_a_tcp_kernel" if stats[-1].get("tc_kernel") == 2 else "phase_a_tc_kernel",
                         "launches": pa_n, "avg_launch_us": pa_ms * 1e3 / max(pa_n, 1),
                         "algorithmic_flops_per_launch": flops / max(pa_n, 1)},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


C3_WORKLOAD = ("differentiable objective: n=1000 dense Q in [-100,100], b in [-50,50], p uniform in [0,100], "
               "64 box points, h and grad h (ubqp_penalized_eval)")


def run_c3(args):
    """The penalized objective and its gradient (the autograd forward) on the 64 C3 points,
    FP32 and FP64: value = gradient entries per second (64 x n per call).  Each call is timed
    with CUDA events on its stream (the entry point's scratch set-up, the GEMV kernel and the
    reduction of h).  Algorithmic bytes: Q once per call plus the points and gradients; the
    kernel reads Q once per point, from L2 after the first (reported as l2_bytes_per_call)."""
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    from paper_2408_04875_gb300 import instances as I
    torch.cuda.set_device(0)
    Q, b = I.c3_instance(1000, 1)
    X = I.box_points(1000, 64, 1)
    p = np.random.default_rng(1).uniform(0, 100, 1000)
    peak, peak_kind = _peaks()
    out = {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        Qt, bt, pt, Xt = (torch.tensor(a, dtype=dt, device="cuda") for a in (Q, b, p, X))
        for _ in range(max(args.warmup, 3)):
            ub.penalized_eval(Qt, bt, pt, Xt)
        n_calls = max(args.steps, 1) * 50
        es = 8 if dt == torch.float64 else 4
        ms = []
        for _ in range(n_calls):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ub.penalized_eval(Qt, bt, pt, Xt)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms) * 1e-3
        alg = es * (1000 * 1000 + 3 * 1000 + 2 * 64 * 1000) + es * 64
        out[name] = {"us_per_call": t * 1e6, "value": 64 * 1000 / t, "algorithmic_bytes_per_call": alg,
                     "achieved_gbs": alg / t / 1e9, "frac_hbm": alg / t / 1e9 / peak,
                     "l2_bytes_per_call": 64 * es * 1000 * 1000, "l2_gbs": 64 * es * 1e6 / t / 1e9,
                     "fp_gflops": 2 * 64 * 1e6 / t / 1e9}
    line = {"metric": "penalized objective + gradient entries/s", "value": out["f32"]["value"],
            "unit": "gradient entries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["f32"]["us_per_call"] * 1e-3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": C3_WORKLOAD, "f64": out["f64"], "l2": "Q (4 MB FP32) is L2-resident"},
            "roofline": {"bound": "hbm", "achieved": out["f32"]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": out["f32"]["frac_hbm"], "traffic": None, "kernel": "phase_a_gemv_kernel",
                         "peak_kind": peak_kind, "f32": out["f32"]}}
    print(json.dumps(line), flush=True)
    return 0


PPA_WORKLOAD = ("PPA (Alg. 1) against PABB (Alg. 2) as the subproblem solver: the 10 n=250 and 10 n=500 "
                "instances of the sweep on the FP32 path (one start), and the batched-restart instance at n=1000 "
                "with 32 starts on the BF16 x2 tensor-core path")


def run_ppa(args):
    """The paper compares its two subproblem solvers (Tables 1-5: CPU time and objective).
    Same comparison on the GPU paths: for each solver, the device time of the whole solve, the
    inner iterations (gradient evaluations), the outer steps and the best objectives."""
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    from paper_2408_04875_gb300 import instances as I
    torch.cuda.set_device(0)
    out = {}
    Qs, mus = _instances(0, (250, 500), SEEDS_PER_SIZE)
    Qd = [torch.from_numpy(Q).cuda() for Q in Qs]
    Md = [torch.from_numpy(m).cuda() for m in mus]
    Q4, _ = I.c4_instance(1000, 2)
    M4 = np.diag(np.diag(I.perturbation(Q4, 2)))
    S4 = I.random_starts(1000, 31, 2)
    Q4d, M4d, S4d = (torch.from_numpy(a).cuda() for a in (Q4, M4, S4))
    for name, method in (("pabb", ub.PABB), ("ppa", ub.PPA)):
        ub.solve_batched(Qd[:2], None, Md[:2], method=method, max_outer=2)   # warm
        _, f2, s2 = ub.solve_batched(Qd, None, Md, method=method)
        _, f4, s4 = ub.solve(Q4d, None, mu=M4d, starts=S4d, restarts=32, precision=ub.BF16X2_TC, method=method)
        out[name] = {"fp32_sweep": {"ms": s2["ms_device"], "inner_iters": s2["inner_iters"],
                                    "outer_steps": s2["outer_steps"], "objective_sum": float(np.sum(f2))},
                     "tc_batch_n1000_R32": {"ms": s4["ms_device"], "inner_iters": s4["inner_iters"],
                                            "outer_steps": s4["outer_steps"], "objective": float(f4)}}
    ratio = {k: out["ppa"][k]["ms"] / out["pabb"][k]["ms"] for k in out["ppa"]}
    line = {"metric": "PPA vs PABB device time and objective", "value": ratio["fp32_sweep"],
            "unit": "PPA time / PABB time", "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False,
            "dtype": "f32", "data": "synthetic", "config": {"workload": PPA_WORKLOAD, "results": out,
                                                             "time_ratio": ratio}}
    print(json.dumps(line), flush=True)
    return 0


SYNC_WORKLOAD = ("penalty update every K inner iterations (subproblems capped at K = max_inner): the 10 n=250 and "
                 "10 n=500 instances of the sweep, FP32 path, one start")


def run_sync(args):
    """The paper's closing suggestion (update the penalty in step with the inner iterations),
    read as capping each subproblem at K iterations: objective and device time against K."""
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    torch.cuda.set_device(0)
    Qs, mus = _instances(0, (250, 500), SEEDS_PER_SIZE)
    Qd = [torch.from_numpy(Q).cuda() for Q in Qs]
    Md = [torch.from_numpy(m).cuda() for m in mus]
    ub.solve_batched(Qd[:2], None, Md[:2], max_outer=2)   # warm
    rows = []
    for K in (5, 20, 100, 1000, 10000):
        _, f, st = ub.solve_batched(Qd, None, Md, max_inner=K)
        rows.append({"K": K, "ms": st["ms_device"], "objective_sum": float(np.sum(f)),
                     "inner_iters": st["inner_iters"], "outer_steps": st["outer_steps"],
                     "lanes_capped": st["lanes_capped"]})
    base = rows[-1]
    line = {"metric": "objective and device time against the subproblem cap K", "value": rows[0]["ms"] / base["ms"],
            "unit": "time(K=5) / time(K=10000)", "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False,
            "dtype": "f32", "data": "synthetic", "config": {"workload": SYNC_WORKLOAD, "rows": rows}}
    print(json.dumps(line), flush=True)
    return 0


SINGLE_WORKLOAD = ("plain FP32 path, one lane: C1 (n=50, density 0.1, seed 0) and one n=2500 instance of the "
                   "sweep law (seed 0), whole solves")


def run_single(args):
    """The plain FP32 single-instance path: whole solves of one lane on the single-lane persistent
    kernel (gemv_kernel = 3) and on the lock-step scheduler (gemv_kernel = 1), device time per
    step.  Roofline of the single-lane kernel at n = 2500: algorithmic bytes per step (the sparse
    minimum, 6 B per stored entry + 32 B per row) over the time per step, against HBM (the
    sliced storage of one lane, 3.8 MB, is L2-resident, so the fraction can exceed 1)."""
    import torch
    import paper_2408_04875_gb300 as ub
    from paper_2408_04875_gb300 import instances as I
    torch.cuda.set_device(0)
    peak, peak_kind = _peaks()
    out = {}
    sizes = (50, 2500) if args.sizes == SIZES else tuple(args.sizes)
    for n in sizes:
        Q, _ = I.c2_instance(n, 0)
        mu = I.perturbation(Q, 0)
        Qd, Md = torch.from_numpy(Q).cuda(), torch.from_numpy(mu).cuda()
        for gk in (3, 1):
            for _ in range(max(args.warmup, 1)):
                ub.solve(Qd, None, mu=Md, gemv_kernel=gk, max_outer=2)
            ms, steps, alg, f = [], 0, 0, None
            for _ in range(max(args.steps, 1)):
                _, f, st = ub.solve(Qd, None, mu=Md, gemv_kernel=gk)
                ms.append(st["ms_device"])
                steps, alg = st["ticks"], st["alg_bytes"]
            t = statistics.median(ms)
            out[f"n{n}_k{gk}"] = {"ms": t, "steps": steps, "us_per_step": 1e3 * t / max(steps, 1), "objective": f,
                                  "storage": st["storage"], "alg_bytes_per_step": alg / max(steps, 1),
                                  "achieved_gbs": alg / (t * 1e-3) / 1e9}
    big = out[f"n{max(sizes)}_k3"]
    line = {"metric": "plain FP32 path: device time per step of one lane", "value": big["us_per_step"],
            "unit": "us/step", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": big["ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": {"workload": SINGLE_WORKLOAD, "results": out},
            "roofline": {"bound": "hbm", "achieved": big["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": big["achieved_gbs"] / peak, "traffic": None, "kernel": "solo_lane_kernel",
                         "peak_kind": peak_kind, "l2": "the lane's sliced storage is L2-resident"}}
    print(json.dumps(line), flush=True)
    return 0


TCRAW_WORKLOAD = "raw tensor-core contraction: n=2500 BF16 Q_off (integers), 256 starts as two BF16 terms"


def run_tcraw(args):
    """The batched path's contraction alone (ubqp_tc_matmul_probe: D = A (B_hi + B_lo)^T, no
    solver epilogue) at the batched-restart shape, for profiling.  Prints the host wall time of
    each probe call (which includes its allocation and copies)."""
    import ctypes as C
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    L = ub.lib()
    L.ubqp_tc_matmul_probe.restype = C.c_int
    n, R = 2500, 256
    rng = np.random.default_rng(0)
    A = rng.integers(-100, 101, (n, n)).astype(np.float32)
    A = np.triu(A) + np.triu(A, 1).T
    np.fill_diagonal(A, 0)
    X = rng.random((R, n))

    def bits(a):
        t = torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16)
        return t.view(torch.int16).numpy().view(np.uint16).copy(), t.float().numpy()

    Ab, _ = bits(A)
    hb, hf = bits(X)
    lb, _ = bits(X - hf)
    D = np.zeros((R, n), np.float32)
    walls = []
    for _ in range(max(args.steps, 1) + max(args.warmup, 1)):
        t0 = time.perf_counter()
        rc = L.ubqp_tc_matmul_probe(Ab.ctypes.data_as(C.c_void_p), hb.ctypes.data_as(C.c_void_p),
                                    lb.ctypes.data_as(C.c_void_p), C.c_int64(n), C.c_int64(R),
                                    C.c_int32(args.tc_cluster), D.ctypes.data_as(C.c_void_p))
        walls.append((time.perf_counter() - t0) * 1e3)
        if rc != 0:
            print(json.dumps({"workload": TCRAW_WORKLOAD, "error": rc}))
            return 1
    print(json.dumps({"workload": TCRAW_WORKLOAD, "cluster": args.tc_cluster, "wall_ms": walls}), flush=True)
    return 0


C5_WORKLOAD = ("ragged multi-instance batch: 512 instances, n uniform in [100,3000], density uniform in "
               "[0.05,1], half integer-[-100,100] Q, half Max-Cut (+-1 edges, f = -cut), BF16 Q_off on tensor "
               "cores with FP32 accumulation, FP64 exact evaluation, starts per instance from the restart tuner")


def run_c5(args):
    """Tensor-core path on the ragged 512-instance batch: one call runs every instance x start as
    a lane to the end of Alg. 3; the restart tuner picks the starts per instance (its probes run
    before the timed region).  --max-outer caps the penalty loop (for profiling); throughput
    counts the projected-gradient iterations actually run.  The returned objectives are checked
    for exactness on 64 instances of both kinds."""
    import numpy as np
    import torch
    import paper_2408_04875_gb300 as ub
    from paper_2408_04875_gb300 import instances as I
    torch.cuda.set_device(0)
    specs = I.c5_specs(args.c5_count)
    t0 = time.perf_counter()
    Qd, bd, Qh, bh = [], [], [], []
    for sp in specs:
        Q, b = I.c5_instance(sp)
        Qd.append(torch.from_numpy(Q).cuda())
        bd.append(torch.from_numpy(b).cuda())
        if len(Qh) < 64:         # a sample kept on the host to re-evaluate objectives
            Qh.append(Q)
            bh.append(b)
    gen_s = time.perf_counter() - t0
    max_outer = args.max_outer if args.max_outer is not None else 1000
    kw = dict(precision=ub.BF16X2_TC, max_outer=max_outer, tc_cluster=args.tc_cluster)
    # first call: restart tuner + a full warm-up step
    _, _, st0 = ub.solve_batched(Qd, bd, None, restarts=args.c5_restarts, **kw)
    R = st0["restarts"]
    for _ in range(max(0, args.warmup - 1)):
        ub.solve_batched(Qd, bd, None, restarts=R, **kw)
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    stats, xs, objs = [], None, None
    for _ in range(args.steps):
        xs, objs, st = ub.solve_batched(Qd, bd, None, restarts=R, profile_kernels=0 if args.no_profile else 1, **kw)
        stats.append(st)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    # exactness of the returned objectives on the host sample
    exact = all(float(x.astype(np.float64) @ Q @ x.astype(np.float64) + b @ x) == float(f)
                for Q, b, x, f in zip(Qh, bh, xs, objs))
    work = sum(s["var_updates"] for s in stats)
    pa_ms = sum(s["phase_a_ms"] for s in stats)
    pa_n = sum(s["phase_a_launches"] for s in stats)
    by = sum(s["phase_a_bytes"] for s in stats)
    flops = sum(s["phase_a_flops"] for s in stats)
    peak, peak_kind = _peaks()
    ach = by / (pa_ms * 1e-3) / 1e9 if pa_ms > 0 else None
    line = {"metric": METRIC, "value": work / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x2", "data": "synthetic",
            "config": {"workload": C5_WORKLOAD, "instances": len(specs), "max_outer": max_outer,
                       "restarts_per_instance": R, "restart_probe_us": st0["restart_probe_us"],
                       "lanes": stats[-1]["lanes"], "cluster_size": stats[-1]["cluster_size"],
                       "ticks_per_step": stats[-1]["ticks"], "generation_s": round(gen_s, 1),
                       "objectives_exact_on_sample": exact, "exactness_sample": len(Qh),
                       "lanes_capped": stats[-1]["lanes_capped"], "outer_steps": stats[-1]["outer_steps"],
                       "l2": "BF16 Q_off of the batch (3.4 GB) exceeds L2; no flush"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak if ach else None, "traffic": None,
                         "kernel": "phase_a_tcp_kernel" if stats[-1].get("tc_kernel") == 2 else "phase_a_tc_kernel",
                         "launches": pa_n, "avg_launch_us": pa_ms * 1e3 / max(pa_n, 1),
                         "algorithmic_bytes_per_launch": by / max(pa_n, 1),
                         "tflops": flops / (pa_ms * 1e-3) / 1e12 if pa_ms > 0 else None, "peak_kind": peak_kind},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_model() -> str:
    """The host CPU's model name as lscpu prints it (the machine architecture if lscpu is
    missing or says nothing)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cpu_baseline(budget_s: float = 12.0, threads: int | None = None):
    """The FP64 oracle as it stands, on a bounded sample of the same workload: whole solves of
    the n = 250 instances of the sweep (taken in turn, again from the first when all ten have
    started), instance-parallel on `threads` host threads (default: every core; the oracle is
    plain C called through ctypes, which releases the GIL).  No thread starts a solve once the
    budget has run out; the value counts the solves that finished."""
    import concurrent.futures as cf
    import threading
    import oracle as O
    from paper_2408_04875_gb300 import instances as I
    O.build()
    threads = threads or os.cpu_count() or 1
    todo = []
    for seed in range(SEEDS_PER_SIZE):
        Q, _ = I.c2_instance(250, seed)
        todo.append((250, Q, I.perturbation(Q, seed)))
    lock = threading.Lock()
    state = {"next": 0, "work": 0, "done": 0}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                if time.perf_counter() - t0 > budget_s:
                    return
                n, Q, mu = todo[state["next"] % len(todo)]
                state["next"] += 1
            _, _, st = O.solve(Q, None, mu)
            with lock:
                state["work"] += st["grad_evals"] * n
                state["done"] += 1

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for f in [ex.submit(worker) for _ in range(threads)]:
            f.result()
    dt = time.perf_counter() - t0
    return {"value": state["work"] / dt, "unit": UNIT, "cores": threads, "cpu_model": _cpu_model(), "kind": "oracle",
            "sample": f"{state['done']} whole solves of the 10 n=250 instances of the sweep (in turn), "
                      f"{threads} threads, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    steps, ms = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        b = cpu_baseline(budget_s=10.0)
        if i >= args.warmup:
            steps.append(b)
            ms.append((time.perf_counter() - t0) * 1e3)
    value = statistics.mean(s["value"] for s in steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "impl": "reference",
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_sample": steps[-1]["sample"]},
            "cpu_baseline": {"kind": "oracle", "cores": steps[-1]["cores"], "cpu_model": steps[-1]["cpu_model"],
                             "sample": steps[-1]["sample"], "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2408_04875_gb300 as ub

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    Qs, mus = _instances(rank, args.sizes, args.seeds)
    Qd = [torch.from_numpy(Q).cuda() for Q in Qs]
    Md = [torch.from_numpy(m).cuda() for m in mus]
    torch.cuda.synchronize()
    kw = dict(profile_kernels=0 if args.no_profile else 1, gemv_kernel=args.gemv_kernel,
              lane_budget=args.lane_budget, rows_per_item=args.rows_per_item)
    if args.max_outer is not None:
        kw["max_outer"] = args.max_outer
    for _ in range(args.warmup):
        ub.solve_batched(Qd, None, Md, **kw)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    stats = []
    objs = None
    for _ in range(args.steps):
        _, objs, st = ub.solve_batched(Qd, None, Md, **kw)
        stats.append(st)
    e1.record()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max, work_all = aggregate_ranks(ms, sum(s["var_updates"] for s in stats), dist, "cuda")
    value = work_all / (ms_max * 1e-3)

    # end to end through the public API with host buffers (H2D of Q and mu, D2H of x, f)
    st_e2e, e2e_s = None, None
    if not args.no_e2e:
        t0 = time.perf_counter()
        _, _, st_e2e = ub.solve_batched(Qs, None, mus, **{k: v for k, v in kw.items() if k != "profile_kernels"})
        e2e_s = time.perf_counter() - t0
    h2d = sum(Q.nbytes + m.nbytes for Q, m in zip(Qs, mus))
    d2h = sum(Q.shape[0] for Q in Qs) + 8 * len(Qs)

    # roofline of the dominant kernel (phase-A GEMV), CUDA events around every launch.  The
    # algorithmic bytes are the sparse minimum of every matrix-vector product (the stored
    # off-diagonal entries as 4-byte values with 2-byte column indices, plus 8 vectors of n
    # floats per step); the bytes of the storage the kernel reads give frac_storage
    pa_ms = sum(s["phase_a_ms"] for s in stats)
    pa_n = sum(s["phase_a_launches"] for s in stats)
    pa_bytes = sum(s["phase_a_bytes"] for s in stats)
    alg_bytes = sum(s["alg_bytes"] for s in stats)
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (pa_ms * 1e-3) / 1e9 if pa_ms > 0 else None
    achieved_storage = pa_bytes / (pa_ms * 1e-3) / 1e9 if pa_ms > 0 else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": len(Qs), "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (302 MB of FP32 Q per batch); no flush",
                       "time_to_solution_ms": ms_max / args.steps,
                       "inner_iters_per_step": stats[-1]["inner_iters"], "outer_steps_per_step": stats[-1]["outer_steps"],
                       "ticks_per_step": stats[-1]["ticks"], "best_objectives_first3": [float(v) for v in objs[:3]]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": (TRAFFIC_RATIO[(stats[-1]["gemv_kernel"], stats[-1]["storage"])] * alg_bytes
                                     / max(pa_n, 1) if (stats[-1]["gemv_kernel"], stats[-1]["storage"]) in TRAFFIC_RATIO
                                     and pa_n else None),
                         "kernel": GEMV_KERNELS.get(stats[-1]["gemv_kernel"], "?"), "launches": pa_n,
                         "avg_launch_us": pa_ms * 1e3 / max(pa_n, 1),
                         "algorithmic_bytes_per_launch": alg_bytes / max(pa_n, 1),
                         "algorithmic_bytes": "sparse minimum: per lane-step 6 B x stored off-diagonal entries "
                                              "+ 32 B x n",
                         "storage_bytes_per_launch": pa_bytes / max(pa_n, 1),
                         "achieved_storage": achieved_storage,
                         "frac_storage": (achieved_storage / peak) if achieved_storage else None,
                         "peak_kind": peak_kind},
            "e2e": None if st_e2e is None else {"value": st_e2e["var_updates"] / e2e_s, "unit": UNIT,
                                                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clocks,
        }
        if args.sizes != SIZES or args.seeds != SEEDS_PER_SIZE or args.max_outer is not None:
            line["config"]["workload"] = (f"profiling case: n in {list(args.sizes)} x {args.seeds} seeds, "
                                          f"max_outer={args.max_outer}")
        if not args.no_c4:
            line["config"]["time_to_oracle_objective"] = c4_time_to_objective(local)
        line["cpu_baseline"] = None if args.no_cpu_baseline else cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    # profiling knobs (defaults are the benchmark workload)
    ap.add_argument("--sizes", type=lambda v: tuple(int(x) for x in v.split(",")), default=SIZES)
    ap.add_argument("--seeds", type=int, default=SEEDS_PER_SIZE)
    ap.add_argument("--max-outer", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-c4", action="store_true",
                    help="skip the batched-restart time-to-objective comparison of the default line")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "ppa", "sync", "single", "tcraw"])
    ap.add_argument("--tc-cluster", type=int, default=0,
                    help="CTAs splitting K: tcraw (0 = rule, -1 = persistent kernel); c5 (0 = measured "
                         "tuner, 1 = no split: the persistent kernel when the tiles fill the GPU)")
    ap.add_argument("--c5-count", type=int, default=512, help="instances of the ragged batch")
    ap.add_argument("--c5-restarts", type=int, default=0, help="starts per instance (0 = restart tuner)")
    ap.add_argument("--restarts", type=int, default=256)
    ap.add_argument("--gemv-kernel", type=int, default=0, choices=[0, 1, 2, 3],
                    help="scheduler of the FP32 lanes: 0 library's choice, 1 lock-step, 2 lane loop")
    ap.add_argument("--rows-per-item", type=int, default=0,
                    help="FP32 lanes: matrix rows per work item (0 = library default)")
    ap.add_argument("--lane-budget", type=int, default=0,
                    help="lane loop: steps per lane per launch (0 = library default)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c3":
        return run_c3(args)
    if args.workload == "ppa":
        return run_ppa(args)
    if args.workload == "sync":
        return run_sync(args)
    if args.workload == "single":
        return run_single(args)
    if args.workload == "tcraw":
        return run_tcraw(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.workload == "c5":
        return run_c5(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
