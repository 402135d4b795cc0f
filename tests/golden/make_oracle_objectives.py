"""Writes tests/golden/oracle_objectives.json: the FP64 oracle's best objective (Alg. 3
with Alg. 2, oracle/ubqp_oracle.c) on the seeded instances that the GPU parity tests
compare against at the sizes the benchmark times.  Nothing here runs the CUDA library.

Cases:
- "c2": the plain sweep law (density 0.1, integers in [-100, 100], b = 0, the full
  perturbation of Sec. 3.5 drawn by instances.perturbation), one start (x^0 of Eq. (gamma)):
  n = 250, 500 and 1000, seeds 0-2; n = 2500, seed 0.
- "c4": the restart-batch instance law with the diagonal-only perturbation the tensor-core
  path uses; for each start r the oracle's objective of Alg. 3 run from that start alone
  (r = 0: x^0 of Eq. (gamma); r >= 1: row r-1 of instances.random_starts(n, R-1, seed)).
  n = 1000, seed 2, R = 32; and n = 2500, seed 2, start 0 only.
- "c2d": the "c2" instances with the stored entries changed by about one FP32 rounding,
  mu + 1e-7 Q (E + E^T)/2 with E standard normal from numpy's default_rng(draw): draws 1-16
  at n = 250, 500 and 1000, draws 1-7 at n = 2500.  How far these runs spread shows how much
  the method's end point (which local optimum Alg. 3 reaches) depends on rounding.
- "c4d": the same for the n = 2500 restart-batch instance from x^0 (its diagonal-only
  perturbation plus 1e-7 Q (E + E^T)/2), draws 1-7.
- "c5": four instances of the ragged-batch law (instances.c5_specs(4, seed=7, n_lo=100,
  n_hi=400): two integer-Q, two Max-Cut), diagonal-only perturbation drawn as for "c4"
  with the instance's own seed, R = 8 starts each (start 0 = x^0, then
  instances.random_starts(n, 7, seed)).

An oracle solve takes about 1 s at n = 250, 11 s at n = 500, 3 min at n = 1000 and hours at
n = 2500 on one core, so the cases run in a process pool and the file is rewritten after
each finished case (a later run computes only the cases still missing).  Run from the
repository root:
    python tests/golden/make_oracle_objectives.py [--workers K] [--only c2|c2d|c4|c4d|c5] [--out FILE]
    python tests/golden/make_oracle_objectives.py --merge FILE   # add FILE's cases to the golden file
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_objectives.json")
C4_R = 32


def case_list():
    cases = []
    for n, seeds in ((250, (0, 1, 2)), (500, (0, 1, 2)), (1000, (0, 1, 2)), (2500, (0,))):
        for s in seeds:
            cases.append({"family": "c2", "n": n, "seed": s, "start": 0})
            for d in range(1, (7 if n == 2500 else 16) + 1):
                cases.append({"family": "c2d", "n": n, "seed": s, "start": 0, "draw": d})
    for r in range(C4_R):
        cases.append({"family": "c4", "n": 1000, "seed": 2, "start": r, "R": C4_R})
    cases.append({"family": "c4", "n": 2500, "seed": 2, "start": 0, "R": 256})
    for d in range(1, 8):
        cases.append({"family": "c4d", "n": 2500, "seed": 2, "start": 0, "R": 256, "draw": d})
    from paper_2408_04875_gb300 import instances as I
    for i, (n, dens, kind, s) in enumerate(I.c5_specs(4, seed=7, n_lo=100, n_hi=400)):
        for r in range(8):
            cases.append({"family": "c5", "n": n, "seed": s, "start": r, "R": 8, "index": i, "density": dens,
                          "kind": kind})
    return cases


def key(c):
    k = f"{c['family']}:n={c['n']}:seed={c['seed']}:start={c['start']}"
    return k + f":draw={c['draw']}" if "draw" in c else k


def run_case(c):
    import numpy as np
    import oracle as O
    from paper_2408_04875_gb300 import instances as I
    t0 = time.time()
    if c["family"] in ("c2", "c2d"):
        Q, b = I.c2_instance(c["n"], c["seed"])
        mu = I.perturbation(Q, c["seed"])
        if c["family"] == "c2d":
            E = np.random.default_rng(c["draw"]).standard_normal(Q.shape)
            mu = mu + 1e-7 * Q * (E + E.T) / 2
        xs = None
    else:
        if c["family"] in ("c4", "c4d"):
            Q, b = I.c4_instance(c["n"], c["seed"])
        else:
            Q, b = I.c5_instance((c["n"], c["density"], c["kind"], c["seed"]))
        mu = np.diag(np.diag(I.perturbation(Q, c["seed"])))
        if c["family"] == "c4d":
            E = np.random.default_rng(c["draw"]).standard_normal(Q.shape)
            mu = mu + 1e-7 * Q * (E + E.T) / 2
        xs = None if c["start"] == 0 else I.random_starts(c["n"], c["R"] - 1, c["seed"])[c["start"] - 1]
    x, f, st = O.solve(Q, b, mu, x_start=xs)
    out = dict(c)
    out.update({"f": f, "outer": st["outer"], "grad_evals": st["grad_evals"], "status": st["status"],
                "x": "".join(str(int(v)) for v in x), "cpu_s": round(time.time() - t0, 1)})
    return out


def load(path=PATH):
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {"source": "FP64 oracle (oracle/ubqp_oracle.c), Alg. 3 with Alg. 2, default options",
            "generator": "tests/golden/make_oracle_objectives.py", "cases": {}}


def save(d, path=PATH):
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--only", default=None)
    ap.add_argument("--out", default=PATH)
    ap.add_argument("--merge", default=None)
    ap.add_argument("--small-first", action="store_true", help="start the short solves first")
    args = ap.parse_args()
    if args.merge:
        d = load()
        d["cases"].update(load(args.merge)["cases"])
        save(d)
        print("merged", args.merge, "->", PATH, len(d["cases"]), "cases")
        return
    import oracle as O
    O.build()
    d = load(args.out)
    todo = [c for c in case_list() if key(c) not in d["cases"] and (args.only is None or c["family"] == args.only)]
    todo.sort(key=lambda c: c["n"] if args.small_first else -c["n"])   # by default the long solves first
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        for res in pool.imap_unordered(run_case, todo):
            d = load(args.out)   # re-read: cases merged by another run since the start stay
            d["cases"][key(res)] = res
            save(d, args.out)
            print(key(res), res["f"], res["cpu_s"], "s", flush=True)


if __name__ == "__main__":
    main()
