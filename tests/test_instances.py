"""The seeded input generators against the recipe they state (CPU).

The generators feed both the CUDA path and the oracle, so a wrong law here would pass
every parity test and still measure the wrong workload.  Checked: symmetry, value ranges,
densities within a binomial bound, the Max-Cut mapping f(y) = -cut(y) of Sec. 5.3 by brute
force, the perturbation's support and scale (Sec. 3.6), the ragged-batch law, determinism
per seed, and that the module holds no arithmetic of the method.
"""
import ast
import itertools
import pathlib

import numpy as np
import pytest

from paper_2408_04875_gb300 import instances as I


def _upper_fraction(Q):
    iu = np.triu_indices(Q.shape[0])
    return np.count_nonzero(Q[iu]) / iu[0].size, iu[0].size


@pytest.mark.parametrize("n,density,seed", [(50, 0.1, 0), (250, 0.1, 3), (300, 0.6, 5)])
def test_random_ubqp_law(n, density, seed):
    Q, b = I.random_ubqp(n, density, seed)
    assert Q.dtype == np.float64 and Q.flags.c_contiguous
    assert np.array_equal(Q, Q.T)
    assert np.array_equal(Q, np.round(Q)) and Q.min() >= -100 and Q.max() <= 100
    assert not b.any()
    # a stored entry is nonzero unless its uniform integer draw was 0 (1 in 201)
    p = density * 200 / 201
    frac, m = _upper_fraction(Q)
    assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / m)


def test_random_ubqp_linear_term_and_determinism():
    Q1, b1 = I.random_ubqp(80, 0.2, 9, b_range=(-20, 20))
    Q2, b2 = I.random_ubqp(80, 0.2, 9, b_range=(-20, 20))
    assert np.array_equal(Q1, Q2) and np.array_equal(b1, b2)
    assert np.array_equal(b1, np.round(b1)) and b1.min() >= -20 and b1.max() <= 20 and b1.any()
    Q3, _ = I.random_ubqp(80, 0.2, 10)
    assert not np.array_equal(Q1, Q3)


def test_dense_ubqp_law():
    Q, b = I.c3_instance(200, 1)
    assert np.array_equal(Q, Q.T)
    assert Q.min() >= -100 and Q.max() <= 100 and b.min() >= -50 and b.max() <= 50
    frac, _ = _upper_fraction(Q)
    assert frac > 0.98   # dense: only draws of exactly 0 are missing


def test_maxcut_mapping_is_minus_cut_by_enumeration():
    """Sec. 5.3: Max-Cut with +-1 weights as the 0/1 problem y'Wy - (We)'y = -cut(y)."""
    n = 10
    W, b = I.maxcut_ubqp(n, 0.5, 4)
    assert np.array_equal(W, W.T) and not np.diag(W).any()
    assert set(np.unique(W)) <= {-1.0, 0.0, 1.0}
    assert np.array_equal(b, -W.sum(axis=1))
    for bits in itertools.product((0, 1), repeat=n):
        y = np.array(bits, dtype=np.float64)
        cut = sum(W[i, j] for i in range(n) for j in range(i + 1, n) if bits[i] != bits[j])
        assert y @ W @ y + b @ y == -cut


def test_maxcut_density_and_signs():
    W, _ = I.maxcut_ubqp(400, 0.3, 2)
    iu = np.triu_indices(400, 1)
    e = W[iu]
    m = e.size
    assert abs(np.count_nonzero(e) / m - 0.3) < 5 * np.sqrt(0.3 * 0.7 / m)
    pos = np.count_nonzero(e > 0) / np.count_nonzero(e)
    assert abs(pos - 0.5) < 0.05


def test_perturbation_support_and_scale():
    Q, _ = I.random_ubqp(300, 0.1, 7)
    mu = I.perturbation(Q, 7)
    assert np.array_equal(mu, mu.T)
    off = ~np.eye(300, dtype=bool)
    assert not mu[off & (Q == 0)].any()          # zero off-diagonal entries stay zero
    assert np.all(np.diag(mu) != 0)              # the diagonal is always perturbed
    sigma = 1e-3 * np.abs(Q[off]).max()
    iu = np.triu_indices(300)
    stored = (Q[iu] != 0) | (iu[0] == iu[1])
    z = mu[iu][stored]                           # the independent draws
    assert abs(z.std() / sigma - 1) < 0.05 and abs(z.mean()) < 5 * sigma / np.sqrt(z.size)
    # an empty off-diagonal falls back to sigma = sigma_rel
    mu1 = I.perturbation(np.zeros((1, 1)), 0)
    assert mu1.shape == (1, 1) and 0 < abs(mu1[0, 0]) < 1e-2


def test_starts_and_box_points():
    s = I.random_starts(64, 255, 2)
    p = I.box_points(64, 10, 2)
    assert s.shape == (255, 64) and p.shape == (10, 64)
    assert s.min() >= 0 and s.max() < 1 and p.min() >= 0 and p.max() < 1
    assert not np.array_equal(s[:10], p)         # separate streams


def test_ragged_batch_law():
    specs = I.c5_specs(512)
    assert len(specs) == 512 and specs == I.c5_specs(512)
    ns = np.array([s[0] for s in specs])
    dens = np.array([s[1] for s in specs])
    assert ns.min() >= 100 and ns.max() <= 3000 and np.ptp(ns) > 2500
    assert dens.min() >= 0.05 and dens.max() <= 1.0 and np.ptp(dens) > 0.8
    assert [s[2] for s in specs] == ["int" if i % 2 == 0 else "maxcut" for i in range(512)]
    assert len({s[3] for s in specs}) == 512
    Q, b = I.c5_instance((120, 0.3, "maxcut", 5))
    assert np.array_equal(b, -Q.sum(axis=1))
    Q, b = I.c5_instance((120, 0.3, "int", 5))
    assert not b.any()


def test_generators_hold_no_method_arithmetic():
    """The module imports nothing but numpy (and __future__): neither the library nor the
    oracle, so both sides of a parity test draw from it independently."""
    src = pathlib.Path(I.__file__).read_text()
    mods = set()
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add((node.module or "").split(".")[0] if node.level == 0 else "<relative>")
    assert mods <= {"numpy", "__future__"}, mods
