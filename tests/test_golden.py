"""The stored exhaustive optima and the enumeration that wrote them (CPU).

``tests/golden/bruteforce_n16_n20.json`` holds the exact optimum of the small random
instances; every global-quality check compares against it.  Checked here:
- the enumeration (``oracle/brute.py``, vectorized over chunks of points) against a plain
  double loop over every binary point, written independently, on small instances with
  b != 0 and with ties;
- the stored file against a fresh enumeration of the same seeded instances (all n = 16
  cases and one n = 20 case, so that the file still matches its generator);
- each stored x* attains its stored f* exactly.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle.brute import enumerate_min
from paper_2408_04875_gb300 import instances as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "bruteforce_n16_n20.json")


def _plain_min(Q, b):
    n = Q.shape[0]
    best, arg = None, None
    for bits in itertools.product((0, 1), repeat=n):     # x_0 is the slowest bit here
        f = 0.0
        for i in range(n):
            if bits[i]:
                f += b[i]
                for j in range(n):
                    if bits[j]:
                        f += Q[i, j]
        if best is None or f < best:
            best, arg = f, bits
    return best, arg


@pytest.mark.parametrize("n,seed", [(6, 0), (8, 1), (9, 2), (10, 3)])
def test_enumeration_matches_a_plain_double_loop(n, seed):
    Q, b = I.random_ubqp(n, 0.5, seed, b_range=(-60, 60))
    f, x = enumerate_min(Q, b)
    f_plain, _ = _plain_min(Q, b)
    assert f == f_plain
    xf = x.astype(np.float64)
    assert xf @ Q @ xf + b @ xf == f


def test_enumeration_with_ties_returns_a_minimiser():
    Q = np.zeros((5, 5))                                   # every point has f = 0
    f, x = enumerate_min(Q, np.zeros(5))
    assert f == 0.0 and x.shape == (5,)


def test_stored_optima_match_a_fresh_enumeration():
    cases = json.load(open(GOLD))["cases"]
    assert len(cases) == 20
    for c in cases:
        Q, b = I.random_ubqp(c["n"], 0.1, c["seed"])
        x = np.array([int(ch) for ch in c["x_star"]], dtype=np.float64)
        assert x @ Q @ x + b @ x == c["f_star"]             # the stored point attains it
        if c["n"] == 16 or (c["n"] == 20 and c["seed"] == 0):
            f, _ = enumerate_min(Q, b)
            assert f == c["f_star"], c


OBJ = os.path.join(os.path.dirname(__file__), "golden", "oracle_objectives.json")


def test_stored_oracle_objectives_are_attained_by_their_points():
    """Every stored oracle objective (tests/golden/oracle_objectives.json: the sweep law, its
    rounding draws, the restart and ragged-batch laws and the restart instance's draws) is the
    exact objective of the stored binary point on the stored instance, recomputed here with a
    plain product; every sweep instance has its draws (16, or 7 at n = 2500), and so does the
    n = 2500 restart instance (7)."""
    cases = json.load(open(OBJ))["cases"]
    inst = {}
    for key, c in sorted(cases.items()):
        x = np.array([int(v) for v in c["x"]], dtype=np.float64)
        fam, n, seed = c["family"], c["n"], c["seed"]
        if (fam, n, seed) not in inst:
            if fam in ("c2", "c2d"):
                inst[(fam, n, seed)] = I.c2_instance(n, seed)
            elif fam in ("c4", "c4d"):
                inst[(fam, n, seed)] = I.c4_instance(n, seed)
            else:
                inst[(fam, n, seed)] = I.c5_instance((n, c["density"], c["kind"], seed))
        Q, b = inst[(fam, n, seed)]
        assert x.shape == (n,), key
        f = float(x @ Q @ x + (0.0 if b is None else b @ x))
        assert f == c["f"], (key, f, c["f"])
    for key, c in cases.items():
        if c["family"] == "c2":
            pre = f"c2d:n={c['n']}:seed={c['seed']}:start=0:draw="
            draws = [k for k in cases if k.startswith(pre)]
            assert len(draws) == (7 if c["n"] == 2500 else 16), (key, len(draws))
    assert len([k for k in cases if k.startswith("c4d:n=2500:seed=2:start=0:draw=")]) == 7
