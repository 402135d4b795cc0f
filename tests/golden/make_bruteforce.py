"""Writes tests/golden/bruteforce_n16_n20.json: the exact optimum of the small
single-instance cases (n = 16 and 20, seeds 0-9, density 0.1, integers in
[-100, 100], b = 0) by exhaustive enumeration (oracle/brute.py).

The paper prints no worked example with its data, so these enumerated optima are
the stored pins for the global-quality checks.  Run from the repository root:
    python tests/golden/make_bruteforce.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.brute import enumerate_min  # noqa: E402
from paper_2408_04875_gb300 import instances  # noqa: E402


def main():
    out = {"source": "exhaustive enumeration of all 2^n binary points (oracle/brute.py)",
           "family": "random_ubqp(n, density=0.1, seed), integers in [-100,100], b=0",
           "cases": []}
    for n in (16, 20):
        for seed in range(10):
            Q, b = instances.random_ubqp(n, 0.1, seed)
            f, x = enumerate_min(Q, b)
            out["cases"].append({"n": n, "seed": seed, "f_star": f, "x_star": "".join(map(str, x))})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bruteforce_n16_n20.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
