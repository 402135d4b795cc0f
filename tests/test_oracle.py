"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
exhaustive enumeration, closed forms, the paper's lemmas, library eigenvalues and
finite differences.  Each test names the passage it checks."""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle.brute import enumerate_min
from paper_2408_04875_gb300 import instances as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "bruteforce_n16_n20.json")


def _small(n=12, seed=0, density=0.4):
    Q, b = I.random_ubqp(n, density, seed, b_range=(-50, 50))
    return Q, b


# ---- Eq. (bqp): objective --------------------------------------------------------

def test_objective_matches_maxcut_edge_count():
    """Max-Cut mapping of Sec. 5.3: f(y) must equal minus the number-weighted cut,
    counted edge by edge."""
    W, b = I.maxcut_ubqp(14, 0.5, 3)
    rng = np.random.default_rng(0)
    for _ in range(20):
        y = rng.integers(0, 2, 14).astype(np.uint8)
        cut = sum(W[i, j] for i in range(14) for j in range(i + 1, 14) if y[i] != y[j])
        assert O.objective(W, b, y) == -cut


def test_objective_equals_penalized_on_binary_points():
    """Sec. 2.2 / problem (p): h(x,p) = f(x) for every p when x is binary."""
    Q, b = _small()
    rng = np.random.default_rng(1)
    for _ in range(10):
        x = rng.integers(0, 2, Q.shape[0]).astype(np.uint8)
        p = rng.uniform(-50, 50, Q.shape[0])
        assert O.penalized(Q, b, p, x.astype(float), want_grad=False) == pytest.approx(
            O.objective(Q, b, x), abs=1e-9)


def test_reformulation_leaves_binary_objective_unchanged():
    """Sec. 3.5: Q + Diag(gamma), b - gamma give the same f on {0,1}^n."""
    Q, b = _small(10, 2)
    Qp, bp, gam = O.reformulate(Q, b, None)
    assert np.all(gam > 2 * np.abs(Q).sum(1) + np.abs(b))
    f1, x1 = enumerate_min(Q, b)
    f2, x2 = enumerate_min(Qp, bp)
    assert f1 == f2 and np.array_equal(x1, x2)


def test_reformulation_with_perturbation_is_the_perturbed_objective():
    """Sec. 3.5: the shift Diag(gamma) cancels against b' = b - gamma on binary points while
    the perturbation stays: x'Q'x + b''x = f(x) + x'mu x for every binary x."""
    Q, b = _small(16, 3)
    mu = I.perturbation(Q, 3)
    Qp, bp, _ = O.reformulate(Q, b, mu)
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.integers(0, 2, 16).astype(np.uint8)
        xf = x.astype(np.float64)
        assert O.objective(Qp, bp, x) == pytest.approx(O.objective(Q, b, x) + xf @ mu @ xf, abs=1e-9)


# ---- h and its gradient ----------------------------------------------------------

def test_gradient_matches_central_differences():
    """A quadratic has zero third derivative, so the central difference with step
    1e-3 is exact up to rounding."""
    Q, b = I.dense_ubqp(40, 1)
    rng = np.random.default_rng(2)
    p = rng.uniform(0, 100, 40)
    x = rng.random(40)
    h0, g = O.penalized(Q, b, p, x)
    fd = np.empty(40)
    for i in range(40):
        e = np.zeros(40); e[i] = 1e-3
        fd[i] = (O.penalized(Q, b, p, x + e, False) - O.penalized(Q, b, p, x - e, False)) / 2e-3
    assert np.max(np.abs(fd - g)) <= 1e-7 * np.max(np.abs(g))


def test_lemma_4_1_monotone_in_p():
    """Lemma 4.1: h(x, p1) <= h(x, p2) on the box whenever p1 <= p2."""
    Q, b = _small()
    rng = np.random.default_rng(3)
    for _ in range(50):
        x = rng.random(Q.shape[0])
        p1 = rng.uniform(-100, 100, Q.shape[0])
        p2 = p1 + rng.uniform(0, 100, Q.shape[0])
        assert O.penalized(Q, b, p1, x, False) <= O.penalized(Q, b, p2, x, False) + 1e-9


# ---- Eq. (cret) and rho ----------------------------------------------------------

def test_kkt_residual_index_sets():
    """Sec. 3.3: interior coordinates count |g|, x=0 counts max(-g,0), x=1 counts max(g,0)."""
    x = np.array([0.0, 0.0, 1.0, 1.0, 0.5])
    assert O.kkt_residual(x, np.array([3.0, 0, 0, 0, 0])) == 0.0
    assert O.kkt_residual(x, np.array([-3.0, 0, 0, 0, 0])) == 3.0
    assert O.kkt_residual(x, np.array([0, 0, -4.0, 0, 0])) == 0.0
    assert O.kkt_residual(x, np.array([0, 0, 4.0, 0, 0])) == 4.0
    assert O.kkt_residual(x, np.array([0, 0, 0, 0, -2.5])) == 2.5


def test_rho_hand_example():
    Q = np.array([[2.0, -7.0], [-7.0, 1.0]])
    assert O.rho(Q, np.array([0.0, 0.0]), np.array([0.0, 0.0])) == 14.0
    assert O.rho(Q, np.array([30.0, 0.0]), np.array([0.0, 0.0])) == 30.0
    assert O.rho(Q, np.array([0.0, 0.0]), np.array([-20.0, 0.0])) == 44.0   # |2(2+20)|
    assert O.rho(Q, np.array([30.0, 0.0]), np.array([25.0, 0.0])) == 55.0   # |30+25| > |2(2-25)|
    assert O.rho(np.zeros((1, 1)), np.zeros(1), np.zeros(1)) == 1.0


# ---- Eq. (gamma): x^0 --------------------------------------------------------------

def test_initial_point_solves_first_order_condition_and_is_interior():
    """Sec. 3.5: 2(Q + Diag gamma) x = gamma - b, and gamma as chosen keeps 0 < x < 1."""
    for seed in range(3):
        Q, b = I.random_ubqp(60, 0.3, seed, b_range=(-50, 50))
        mu = I.perturbation(Q, seed)
        Qp, bp, gam = O.reformulate(Q, b, mu)
        x0 = O.initial_point(Qp, bp)
        assert np.max(np.abs(2 * Qp @ x0 + bp)) <= 1e-10 * np.max(gam)
        assert np.all(x0 > 0) and np.all(x0 < 1)
        # x0 - e/2 = -(1/2) Q'^-1 ((Q+mu) e + b) and, Q' being strictly diagonally
        # dominant, ||Q'^-1||_inf <= 1 / min_i (Q'_ii - sum_{j!=i} |Q'_ij|)
        Qm = Q + mu
        off = np.abs(Qp).sum(1) - np.abs(np.diag(Qp))
        bound = 0.5 * np.max(np.abs(Qm.sum(1) + b)) / np.min(np.diag(Qp) - off)
        assert np.max(np.abs(x0 - 0.5)) <= bound * (1 + 1e-12)


# ---- lambda_min ------------------------------------------------------------------

@pytest.mark.parametrize("m", [1, 2, 3, 7, 40, 130])
def test_lambda_min_matches_library_eigvalsh(m):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, m))
    A = A + A.T + np.diag(rng.uniform(-3, 3, m))
    assert O.lambda_min(A) == pytest.approx(np.linalg.eigvalsh(A)[0], rel=1e-12, abs=1e-12)


def test_lambda_min_closed_forms():
    a, c, d = 3.0, -1.5, 0.5
    lam = (a + d) / 2 - np.sqrt(((a - d) / 2) ** 2 + c * c)
    assert O.lambda_min(np.array([[a, c], [c, d]])) == pytest.approx(lam, rel=1e-14)
    assert O.lambda_min(np.diag([4.0, -2.0, 9.0])) == pytest.approx(-2.0, rel=1e-14)


def test_penalty_step_first_outer_step_positive():
    """At s = 0, p = 0 and Q' is strictly diagonally dominant: lambda > 0 (Sec. 3.4)."""
    Q, b = I.random_ubqp(50, 0.1, 0)
    mu = I.perturbation(Q, 0)
    Qp, bp, _ = O.reformulate(Q, b, mu)
    x0 = O.initial_point(Qp, bp)
    a, m, lam, fb = O.penalty_step(Qp, bp, np.zeros(50), x0)
    z = x0 - x0 ** 2
    ref = np.linalg.eigvalsh(Qp / np.sqrt(np.outer(z, z)))[0]
    assert m == 50 and not fb and lam > 0
    assert lam == pytest.approx(ref, rel=1e-10) and a == pytest.approx(0.9 * ref, rel=1e-10)


def test_penalty_step_with_penalty_and_boundary_coordinates():
    """Eq. (eq:alpha): lambda_min of Z^-1/2 (Q' - P*)_II Z^-1/2 over the interior set I only;
    coordinates at 0 or 1 drop out, and the current penalty enters the matrix."""
    Q, b = I.random_ubqp(40, 0.2, 3)
    Qp, bp, _ = O.reformulate(Q, b, I.perturbation(Q, 3))
    x = O.initial_point(Qp, bp)
    x[0], x[1] = 0.0, 1.0
    p = 0.2 * np.diag(Qp)
    a, m, lam, fb = O.penalty_step(Qp, bp, p, x)
    z = (x - x ** 2)[2:]
    Qb = (Qp - np.diag(p))[2:, 2:]
    ref = np.linalg.eigvalsh(Qb / np.sqrt(np.outer(z, z)))[0]
    assert m == 38 and not fb
    assert lam == pytest.approx(ref, rel=1e-10) and a == pytest.approx(0.9 * ref, rel=1e-10)


def test_penalty_floor_doubles_per_consecutive_step():
    """The floor reading: with no usable curvature (lambda_min < 0 here, checked against the
    library) the step is positive, doubles for every consecutive floor step, and stops
    doubling after 60."""
    Q, b = I.random_ubqp(30, 0.3, 5)
    Qp, bp, _ = O.reformulate(Q, b, None)
    x = O.initial_point(Qp, bp)
    p = 3.0 * np.diag(Qp)
    z = x - x ** 2
    ref = np.linalg.eigvalsh((Qp - np.diag(p)) / np.sqrt(np.outer(z, z)))[0]
    a0, _, lam, fb = O.penalty_step(Qp, bp, p, x)
    assert ref < 0 and lam == pytest.approx(ref, rel=1e-10) and fb and a0 > 0
    for c in range(1, 6):
        a, _, _, fbc = O.penalty_step(Qp, bp, p, x, consecutive=c)
        assert fbc and a == a0 * 2 ** c
    assert O.penalty_step(Qp, bp, p, x, consecutive=61)[0] == O.penalty_step(Qp, bp, p, x, consecutive=60)[0]


def test_penalty_update_shrinks_scaled_curvature_by_one_minus_eta():
    """Lemma 3.1 with Eq. (pp1): after p <- p + alpha z with alpha = eta lambda_min, the
    matrix Z^-1/2 (Q' - P*) Z^-1/2 is the old one shifted by -alpha I, so its smallest
    eigenvalue is (1 - eta) times the old one (library eigenvalues, one outer step)."""
    Q, b = I.random_ubqp(40, 0.2, 6)
    mu = I.perturbation(Q, 6)
    Qp, bp, _ = O.reformulate(Q, b, mu)
    x0 = O.initial_point(Qp, bp)
    _, _, st = O.solve(Q, b, mu, o=O.opts(max_outer=1))
    assert st["outer"] == 1
    p = st["p"]
    S = 1.0 / np.sqrt(np.outer(x0 - x0 ** 2, x0 - x0 ** 2))
    lam0 = np.linalg.eigvalsh(Qp * S)[0]
    lam1 = np.linalg.eigvalsh((Qp - np.diag(p)) * S)[0]
    assert lam0 > 0 and lam1 == pytest.approx(0.1 * lam0, rel=1e-9)


# ---- Alg. 2 / Alg. 1 ---------------------------------------------------------------

def _equal_curvature_case(n=6, c=3.0, seed=12):
    """Q' = Diag(d), p = d - c: every coordinate has curvature c; the box minimiser of
    h(., p) is clip(t) with t drawn first and b' chosen to make it so."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(5, 10, n)
    p = d - c
    t = rng.uniform(-0.4, 1.4, n)
    bp = -2 * c * t - p
    return np.diag(d), bp, p, np.clip(t, 0, 1), rng.uniform(0.2, 0.8, n)


def test_pabb_first_step_is_the_newton_step_at_equal_curvature():
    """Alg. 2: alpha_0 = 1 / (2 ||Q' - P*||_inf); when every coordinate has the same
    curvature c that is 1 / (2c), the Newton step, so the first projected step lands on
    the box minimiser and the KKT test stops the loop."""
    Qp, bp, p, xs, x0 = _equal_curvature_case()
    r = O.inner(Qp, bp, p, x0, trace_len=3)
    assert r["steps"] == 1 and r["exit"] == 0
    assert np.max(np.abs(r["x"] - xs)) <= 1e-13


def test_ppa_step_is_exact_on_a_diagonal_problem():
    """Alg. 1 with h_p of Sec. 3.1: for diagonal Q' > P* the proximal weight h_p = Q'_ii - p_i
    equals the curvature, so one step reaches the box minimiser."""
    rng = np.random.default_rng(13)
    n = 8
    d = rng.uniform(2, 9, n)
    p = rng.uniform(0, 0.5, n) * d
    t = rng.uniform(-0.5, 1.5, n)
    bp = -2 * (d - p) * t - p
    r = O.inner(np.diag(d), bp, p, rng.uniform(0.2, 0.8, n), O.opts(method=1))
    assert r["steps"] == 1 and r["exit"] == 0
    assert np.max(np.abs(r["x"] - np.clip(t, 0, 1))) <= 1e-13


def test_pabb_separable_case_reaches_closed_form():
    """Q_off = 0: h is separable and strictly convex on the box when Q_ii - p_i > 0;
    its minimiser is clip(-bbar_i / (2 Qbar_ii), 0, 1)."""
    rng = np.random.default_rng(5)
    n = 30
    d = rng.uniform(1, 10, n)
    Qp = np.diag(d)
    bp = rng.uniform(-30, 30, n)
    p = rng.uniform(0, 0.5, n)
    r = O.inner(Qp, bp, p, np.full(n, 0.5), O.opts(tol_inner=1e-12))
    xs = np.clip(-(bp + p) / (2 * (d - p)), 0, 1)
    assert r["exit"] in (0, 2)
    assert np.max(np.abs(r["x"] - xs)) <= 1e-9


def test_iterates_stay_in_box_and_steps_positive():
    Q, b = I.random_ubqp(50, 0.1, 1)
    Qp, bp, _ = O.reformulate(Q, b, I.perturbation(Q, 1))
    x0 = O.initial_point(Qp, bp)
    p = np.full(50, 0.5) * np.diag(Qp)
    r = O.inner(Qp, bp, p, x0, trace_len=200)
    tx = r["trace_x"][: min(200, r["steps"] + 1)]
    assert np.all(tx >= 0.0) and np.all(tx <= 1.0)
    ta = r["trace_alpha"][: min(200, r["steps"])]
    assert np.all(ta > 0)


def test_bb_steps_follow_alternation():
    """Eq. (bb1): odd k uses s^T s / s^T y, even k uses s^T y / y^T y of the last pair."""
    Q, b = I.random_ubqp(40, 0.3, 4)
    Qp, bp, _ = O.reformulate(Q, b, None)
    x0 = O.initial_point(Qp, bp)
    p = 0.3 * np.diag(Qp)
    r = O.inner(Qp, bp, p, x0, trace_len=30)
    X, A = r["trace_x"], r["trace_alpha"]
    Qb = Qp - np.diag(p)
    for k in range(1, min(25, r["steps"])):
        s = X[k] - X[k - 1]
        y = 2 * Qb @ s
        if s @ y <= 0:
            continue
        want = (s @ s) / (s @ y) if k % 2 == 1 else (s @ y) / (y @ y)
        assert A[k] == pytest.approx(want, rel=1e-9)


def test_lemma_4_2_large_penalty_gives_binary_points():
    """Lemma 4.2 / Thm 4.3: with p > diag(Q) every local minimiser is binary, so the
    subproblem solver started anywhere stops at a binary point."""
    Q, b = I.random_ubqp(16, 0.3, 7)
    Qp, bp, _ = O.reformulate(Q, b, None)
    p = np.diag(Qp) + 1.0
    rng = np.random.default_rng(7)
    for _ in range(10):
        r = O.inner(Qp, bp, p, rng.random(16))
        assert np.all((r["x"] == 0.0) | (r["x"] == 1.0))


def test_theorem_4_3_box_minimum_not_below_binary_optimum():
    """Lemma 4.1 with Thm 4.3: min over the box of h(., p) <= min f, with equality once
    p > diag(Q); sampled box points never go below f* then."""
    Q, b = I.random_ubqp(14, 0.4, 8, b_range=(-20, 20))
    fstar, _ = enumerate_min(Q, b)
    p = np.diag(Q) + 1.0
    X = np.random.default_rng(8).random((20000, 14))
    H = np.einsum("ij,jk,ik->i", X, Q, X) + X @ b + ((X - X * X) * p).sum(1)
    assert H.min() >= fstar - 1e-9


def test_ppa_descent_lemma_4_4():
    """Lemma 4.4: h(x^{k+1}) <= h(x^k) - d^T (H_p - Q + P*) d along Alg. 1, and
    H_p + P is positive semidefinite (Sec. 3.1)."""
    Q, b = I.random_ubqp(40, 0.3, 9)
    Qp, bp, _ = O.reformulate(Q, b, I.perturbation(Q, 9))
    x0 = O.initial_point(Qp, bp)
    p = 0.7 * np.diag(Qp)
    o = O.opts(method=1)
    r = O.inner(Qp, bp, p, x0, o, trace_len=60)
    r_abs = np.abs(Qp).sum(1)
    hp = np.maximum(r_abs - p, 1e-8 * max(1.0, r_abs.max()))
    M = np.diag(hp) - Qp + np.diag(p)
    assert np.linalg.eigvalsh(M)[0] >= -1e-9 * np.abs(M).max()
    X = r["trace_x"][: min(60, r["steps"] + 1)]
    for k in range(len(X) - 1):
        d = X[k + 1] - X[k]
        h0 = O.penalized(Qp, bp, p, X[k], False)
        h1 = O.penalized(Qp, bp, p, X[k + 1], False)
        assert h1 <= h0 - d @ M @ d + 1e-8 * abs(h0)


# ---- Alg. 3 ------------------------------------------------------------------------

def test_solve_never_below_enumerated_optimum_and_mostly_reaches_it():
    """Global quality: the rounded objective is never below the exhaustive optimum
    (tests/golden), is exactly f(x_best), and the mean gap stays small (Table 2
    reports 0.06% at n = 20 on the paper's own instances)."""
    cases = json.load(open(GOLD))["cases"]
    gaps = []
    for c in cases:
        Q, b = I.random_ubqp(c["n"], 0.1, c["seed"])
        xb, f, st = O.solve(Q, b, I.perturbation(Q, c["seed"]))
        assert f >= c["f_star"]
        assert f == O.objective(Q, b, xb)
        gaps.append(abs(f - c["f_star"]) / abs(c["f_star"]))
    assert np.mean(gaps) < 0.01
    assert sum(g == 0 for g in gaps) >= 15


def test_solve_terminates_at_binary_point():
    Q, b = I.c1_instance()
    xb, f, st = O.solve(Q, b, I.perturbation(Q, 0))
    assert st["status"] == 0 and st["final_binarity"] <= 1e-5
    assert st["outer"] < 1000
    assert np.all(np.asarray(st["inner_hist"]) <= 10000)


def test_solve_random_start_path():
    Q, b = I.random_ubqp(18, 0.2, 11)
    xs = I.random_starts(18, 1, 11)[0]
    fstar, _ = enumerate_min(Q, b)
    xb, f, st = O.solve(Q, b, I.perturbation(Q, 11), x_start=xs)
    assert f >= fstar and st["status"] == 0


def test_rounding_model_is_off_by_default_and_bounded_when_on():
    """The oracle's FP32 rounding model (fp32_noise, a sensitivity tool for the GPU tests) does
    not touch the arithmetic when off, whatever its seed; when on, the first projected step of
    Alg. 2 moves by at most alpha_0 * 2^-24 * s_i (s_i the gradient's terms) plus one ulp of
    the iterate, and differs between seeds."""
    rng = np.random.default_rng(3)
    n = 40
    Q, b = I.random_ubqp(n, 0.3, 3)
    Qp, bp, _ = O.reformulate(Q, b, I.perturbation(Q, 3))
    x0 = O.initial_point(Qp, bp)
    a, _, _, _ = O.penalty_step(Qp, bp, np.zeros(n), x0)
    p = a * (x0 - x0 * x0)
    x = rng.uniform(0.2, 0.8, n)
    ref = O.inner(Qp, bp, p, x, trace_len=3)
    o = O.opts()
    o.noise_seed = 99
    same = O.inner(Qp, bp, p, x, o, trace_len=3)
    assert np.array_equal(same["trace_x"], ref["trace_x"]) and same["steps"] == ref["steps"]
    d = np.diag(Qp)
    s = 2 * (np.abs(Qp - np.diag(d)) @ np.abs(x)) + np.abs((d - p) * (2 * x - 1)) + np.abs(d + bp)
    alpha0 = 1.0 / (2 * np.max(np.sum(np.abs(Qp - np.diag(p)), axis=1)))
    steps = []
    for seed in (1, 2):
        o.fp32_noise = 2.0 ** -24
        o.noise_seed = seed
        got = O.inner(Qp, bp, p, x, o, trace_len=3)
        dx = np.abs(got["trace_x"][1] - ref["trace_x"][1])
        assert np.all(dx <= alpha0 * 2.0 ** -24 * s + 2.0 ** -23 * np.abs(ref["trace_x"][1]) + 1e-300)
        steps.append(got["trace_x"][1])
    assert not np.array_equal(steps[0], steps[1])
