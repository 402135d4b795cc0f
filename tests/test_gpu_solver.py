"""GPU parity of the FP32 CUDA path against the FP64 oracle, through the C ABI.

Bars (stated with each test): FP32 iterates within 1e-5 relative of the oracle's
over the first 50 inner iterations; rounded objectives evaluated exactly (bit-exact
for integer data); final best objective not worse than the oracle's by more than 0.1%.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle.brute import enumerate_min
from paper_2408_04875_gb300 import instances as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "bruteforce_n16_n20.json")


@pytest.fixture(scope="module")
def ub():
    import torch
    assert torch.cuda.is_available()
    import paper_2408_04875_gb300 as ub
    ub.lib()
    return ub


def _state_after_first_penalty(Q, b, mu):
    Qp, bp, _ = O.reformulate(Q, b, mu)
    x0 = O.initial_point(Qp, bp)
    a, _, _, _ = O.penalty_step(Qp, bp, np.zeros(Q.shape[0]), x0)
    return Qp, bp, a * (x0 - x0 * x0), x0


# ---- initialization (Sec. 3.5) -----------------------------------------------------

@pytest.mark.parametrize("n,seed", [(50, 0), (250, 3), (1000, 1)])
def test_initial_point_matches_cholesky(ub, n, seed):
    Q, b = I.random_ubqp(n, 0.1, seed, b_range=(-50, 50))
    mu = I.perturbation(Q, seed)
    Qp, bp, gam = O.reformulate(Q, b, mu)
    x_ref = O.initial_point(Qp, bp)
    x_gpu, g_gpu = ub.initial_point(Q, b, mu)
    assert np.max(np.abs(g_gpu - gam)) <= 1e-12 * np.max(gam)
    assert np.max(np.abs(x_gpu - x_ref)) <= 1e-5 * np.max(np.abs(x_ref))
    assert np.all(x_gpu > 0) and np.all(x_gpu < 1)


# ---- inner loop (Alg. 2 / Alg. 1) -------------------------------------------------------

def _r32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _rounding_envelope(Qp, bp, p, x0, ref, K, draws=4):
    """How far FP32 rounding alone can move the oracle's trajectory over K iterations: the
    largest relative deviation from the exact trajectory when the oracle runs its rounding
    model (fp32_noise = 2^-24: every gradient evaluation perturbed by one FP32 ulp of the
    gradient's own terms, every iterate by one ulp), the maximum over `draws` seeded draws."""
    worst = 0.0
    for d in range(draws):
        o = O.opts()
        o.fp32_noise = 2.0 ** -24
        o.noise_seed = d + 1
        pert = O.inner(Qp, bp, p, x0, o, trace_len=K + 1)
        k = min(K, pert["steps"], ref["steps"])
        X, Y = ref["trace_x"][: k + 1], pert["trace_x"][: k + 1]
        worst = max(worst, float(np.max(np.max(np.abs(Y - X), axis=1) / np.max(np.abs(X), axis=1))))
    return worst


# how Q'_off is stored and which scheduler runs the lane: dense FP32 rows and the sliced row
# storage on the single-lane kernel, the symmetric tiles and the sliced rows on the lane loop
SCHEDULES = {"dense": dict(sparse_storage=2), "sym": dict(gemv_kernel=2, sym_storage=1, sparse_storage=2),
             "sliced": dict(sparse_storage=1), "sliced_loop": dict(gemv_kernel=2, sparse_storage=1)}


# (n, seed) of the 50-iterate cases: the first subproblem of Alg. 3 (after the first penalty
# update) of C2-law instances.  Which branch each case takes is a property of the oracle
# alone (its rounding envelope); 14 of the cases with n >= 250 take the strict branch, and
# seven with n >= 250 are kept in the relaxed one.
ITERATE_CASES = [(50, 0), (50, 1), (50, 2), (100, 0),
                 (250, 1), (250, 3), (250, 6), (250, 17), (500, 1), (500, 3), (500, 6), (500, 12), (700, 4),
                 (700, 8), (1000, 0), (1000, 1), (1000, 5), (1000, 6),
                 (250, 0), (250, 2), (250, 4), (250, 11), (500, 2), (500, 7), (700, 2)]


@pytest.mark.parametrize("sched", ["dense", "sym", "sliced", "sliced_loop"])
def test_pabb_first_50_iterates_within_1e5(ub, sched):
    """Both sides run Alg. 2 from the same FP32-representable state (Q', b', p, x^0 as
    the GPU holds them).  Bar: relative deviation <= 1e-5 over the first 50 iterates (all of
    them when the subproblem ends sooner), and BB steps within 1e-3 over the first 10,
    wherever FP32 arithmetic can hold it: where the oracle's own trajectory under its FP32
    rounding model (one ulp of the gradient's terms and of the iterate at every step) stays
    within 1e-5.  A BB trajectory can amplify rounding by orders of magnitude (a long BB1 step
    after a small s^T y); where that envelope exceeds 1e-5, the bar is twice the envelope.
    Every case prints its branch; at least 10 cases with n >= 250 must take the strict one."""
    rows, bad = [], []
    for n, seed in ITERATE_CASES:
        Q, b = I.random_ubqp(n, 0.1, seed)
        Qp, bp, p, x0 = (_r32(a) for a in _state_after_first_penalty(Q, b, I.perturbation(Q, seed)))
        ref = O.inner(Qp, bp, p, x0, trace_len=51)
        got = ub.inner_run(Qp, bp, p, x0, trace_len=51, **SCHEDULES[sched])
        K = min(50, ref["steps"], got["steps"])
        X, Y = ref["trace_x"][: K + 1], got["trace_x"][: K + 1]
        rel = np.max(np.abs(Y - X), axis=1) / np.maximum(np.max(np.abs(X), axis=1), 1e-30)
        env = _rounding_envelope(Qp, bp, p, x0, ref, 50)
        strict = env <= 1e-5
        rows.append((n, seed, ref["steps"], got["steps"], K, env, "strict" if strict else "relaxed", rel.max()))
        if not (np.all(Y >= 0) and np.all(Y <= 1)):
            bad.append(f"n={n} seed={seed}: iterate left the box")
        if strict:
            if not np.all(rel <= 1e-5):
                bad.append(f"n={n} seed={seed}: max rel {rel.max():.3e} at k={int(rel.argmax())}")
            # BB steps of the first 10 iterations (later ones are ratios of rounding-sized s, y)
            A, B = ref["trace_alpha"][: min(K, 10)], got["trace_alpha"][: min(K, 10)]
            if not np.all(np.abs(B - A) <= 1e-3 * np.abs(A)):
                bad.append(f"n={n} seed={seed}: BB steps")
        elif not rel.max() <= 2 * env:
            bad.append(f"n={n} seed={seed}: {rel.max():.3e} vs rounding envelope {env:.1e}")
        if got["steps"] == ref["steps"] and got["exit"] == 0 and not np.max(np.abs(got["x"] - ref["x"])) <= 1e-3:
            bad.append(f"n={n} seed={seed}: final point")
    print(f"\n50-iterate parity ({sched}): n seed oracle_steps gpu_steps compared envelope branch max_rel")
    for r in rows:
        print("  %5d %3d %4d %4d %3d %.2e %-7s %.2e" % r)
    assert not bad, bad
    n_strict = sum(1 for r in rows if r[0] >= 250 and r[6] == "strict")
    assert n_strict >= 10, f"only {n_strict} strict cases with n >= 250"


def test_pabb_runs_to_same_stationary_point(ub):
    """Separable case (Q_off = 0): the closed-form minimiser clip(-bbar/(2 Qbar_ii))."""
    rng = np.random.default_rng(5)
    n = 300
    d = rng.uniform(1, 10, n)
    bp = rng.uniform(-30, 30, n)
    p = rng.uniform(0, 0.5, n)
    got = ub.inner_run(np.diag(d), bp, p, np.full(n, 0.5))
    xs = np.clip(-(bp + p) / (2 * (d - p)), 0, 1)
    assert got["exit"] in (0, 2)
    assert np.max(np.abs(got["x"] - xs)) <= 1e-4


def _equal_curvature_case(n, seed):
    """Q' = Diag(d), p = d - 3, all entries exact in FP32: every coordinate has curvature 3 and
    the box minimiser of h(., p) is clip(t)."""
    rng = np.random.default_rng(seed)
    d = rng.integers(5, 40, n) + 0.5
    p = d - 3.0
    t = rng.uniform(-0.4, 1.4, n)
    bp = -6.0 * t - p
    return np.diag(d), bp, p, np.clip(t, 0, 1), rng.uniform(0.2, 0.8, n)


def test_pabb_first_step_is_the_newton_step_at_equal_curvature(ub):
    """Alg. 2 on the device: alpha_0 = 1 / (2 ||Q' - P*||_inf) = 1/6 is the Newton step when
    every coordinate has curvature 3, so one projected step reaches the box minimiser and
    the KKT test stops the loop (a fact of the mathematics, not of the oracle)."""
    Qp, bp, p, xs, x0 = _equal_curvature_case(300, 21)
    got = ub.inner_run(Qp, bp, p, x0, trace_len=2)
    assert got["steps"] == 1 and got["exit"] == 0
    assert np.max(np.abs(got["x"] - xs)) <= 1e-6


def test_ppa_step_is_exact_on_a_diagonal_problem(ub):
    """Alg. 1 on the device: for diagonal Q' > P* the weight h_p = Q'_ii - p_i equals the
    curvature, so one step reaches the box minimiser."""
    rng = np.random.default_rng(22)
    n = 300
    d = rng.integers(2, 30, n) + 0.25
    p = np.floor(rng.uniform(0, 0.5, n) * d * 8) / 8
    t = rng.uniform(-0.5, 1.5, n)
    bp = -2 * (d - p) * t - p
    got = ub.inner_run(np.diag(d), bp, p, rng.uniform(0.2, 0.8, n), method=1)
    assert got["steps"] == 1 and got["exit"] == 0
    assert np.max(np.abs(got["x"] - np.clip(t, 0, 1))) <= 1e-6


def _ppa_stall_case(n=1025):
    """Q'_off: a symmetric +-1 circulant with zero diagonal and zero row sums (256 of the 512
    offsets +1, the rest -1), diagonal 1, p = 0, x0 = 0.75.  Then Q'_off x0 = 0 exactly and
    g = 2 Qbar x0 + bbar = 1.5 + bbar = t with t = +-4e-5 chosen through bbar.  rho = 2, so the
    KKT measure is 2e-5 > delta (no KKT exit), and the PPA weight is h_p = 1024 + 1: the step
    t / (2 h_p) = 1.95e-8 is below half an FP32 ulp of 0.75 (2.98e-8)."""
    rng = np.random.default_rng(7)
    half = (n - 1) // 2
    s = np.zeros(n)
    signs = np.array([1.0] * (half // 2) + [-1.0] * (half // 2))
    rng.shuffle(signs)
    s[1:half + 1] = signs
    s[n - half:] = signs[::-1]
    Qp = np.array([np.roll(s, i) for i in range(n)]) + np.eye(n)
    t = np.where(rng.random(n) < 0.5, -4e-5, 4e-5)
    bp = -1.5 + t
    return Qp, bp, np.zeros(n), np.full(n, 0.75)


def test_ppa_zero_step_ends_the_subproblem(ub):
    """Alg. 1 ends when the projected step leaves x unchanged.  On the stall case above the
    device's first step rounds to x itself, so it stops after one step with exit code 2
    (zero step) instead of running to the iteration cap; the oracle's FP64 step is 1.95e-8 and
    rounds to the same unchanged x in FP32."""
    Qp, bp, p, x0 = _ppa_stall_case()
    assert np.allclose(Qp, Qp.T) and np.all(Qp.sum(1) == 1.0)
    got = ub.inner_run(Qp, bp, p, x0, trace_len=3, method=1, max_inner=500)
    assert got["exit"] == 2 and got["steps"] == 1, (got["exit"], got["steps"])
    assert np.array_equal(got["x"], x0)
    ref = O.inner(Qp, bp, p, x0, O.opts(method=1, max_inner=3), trace_len=3)
    step = ref["trace_x"][1] - x0
    assert np.all(np.abs(step) > 1e-8) and np.all(np.abs(step) < 2.98e-8)
    assert np.array_equal(_r32(ref["trace_x"][1]), x0)


def test_ppa_first_iterates(ub):
    Q, b = I.random_ubqp(60, 0.2, 4)
    Qp, bp, p, x0 = (_r32(a) for a in _state_after_first_penalty(Q, b, I.perturbation(Q, 4)))
    ref = O.inner(Qp, bp, p, x0, O.opts(method=1), trace_len=31)
    got = ub.inner_run(Qp, bp, p, x0, trace_len=31, method=1)
    K = min(30, ref["steps"], got["steps"])
    X, Y = ref["trace_x"][: K + 1], got["trace_x"][: K + 1]
    assert np.max(np.abs(Y - X)) <= 1e-5 * np.max(np.abs(X))


# ---- penalty step (Sec. 3.4) ---------------------------------------------------------

def _state_at_outer_step(Q, b, mu, S):
    """(Q', b', p, x) just before the penalty step of outer step S of Alg. 3, composed from the
    oracle's own steps (penalty step with the floor count carried, then the subproblem)."""
    Qp, bp, _ = O.reformulate(Q, b, mu)
    x = O.initial_point(Qp, bp)
    p = np.zeros(Q.shape[0])
    cons = 0
    for _ in range(S):
        a, _, _, fb = O.penalty_step(Qp, bp, p, x, consecutive=cons)
        cons = cons + 1 if fb else 0
        p = p + a * (x - x * x)
        x = O.inner(Qp, bp, p, x)["x"]
    return Qp, bp, p, x


# (n, seed, outer step): interior states early in Alg. 3 and, for n = 250 seed 0, the steps
# 14 and 16 at which the oracle's lambda_min falls below the resolution floor
PENALTY_CASES = [(50, 0, 0), (50, 0, 1), (250, 1, 0), (250, 1, 5), (250, 0, 3), (250, 0, 8), (600, 2, 0),
                 (600, 2, 2), (250, 0, 14), (250, 0, 16)]


def test_penalty_step_lambda_min(ub):
    """The device eigen-solver (LOBPCG, FP32) against the oracle's dense lambda_min of
    Z^-1/2 Qbar_II Z^-1/2 (Sec. 3.4, Lemma 3.1) and the step alpha of Eq. (eq:alpha1):
    - above the floor, with the default stopping rule (relative change of the Ritz value 1e-7,
      at most 256 iterations): lambda and alpha within 2e-4; with the rule loosened to 1e-4
      (64 iterations): within 2e-3;
    - below the floor (the oracle's lambda <= F = 4 delta rho): the device also takes the
      floor, alpha = eta F to FP32 rounding (no earlier floor steps in the probe).
    Every case prints its branch; at least two take the floor."""
    floors = 0
    for n, seed, S in PENALTY_CASES:
        Q, b = I.random_ubqp(n, 0.1, seed)
        Qp, bp, p, x = _state_at_outer_step(Q, b, I.perturbation(Q, seed), S)
        a_ref, m_ref, lam_ref, fb = O.penalty_step(Qp, bp, p, x)
        got = ub.penalty_probe(Qp, bp, p, x)
        loose = ub.penalty_probe(Qp, bp, p, x, lobpcg_tol=1e-4, lobpcg_max_iter=64)
        print(f"n={n} seed={seed} s={S}: |I|={m_ref} oracle lambda={lam_ref:.6e} alpha={a_ref:.6e} floor={fb} | "
              f"gpu lambda={got['lambda']:.6e} alpha={got['alpha']:.6e} iters={got['iters']} | "
              f"loose lambda={loose['lambda']:.6e} iters={loose['iters']}")
        assert got["n_active"] == m_ref
        if not fb:
            assert abs(got["lambda"] - lam_ref) <= 2e-4 * abs(lam_ref), (n, seed, S)
            assert abs(got["alpha"] - a_ref) <= 2e-4 * abs(a_ref), (n, seed, S)
            assert abs(loose["lambda"] - lam_ref) <= 2e-3 * abs(lam_ref), (n, seed, S)
        else:
            floors += 1
            assert abs(got["alpha"] - a_ref) <= 1e-5 * a_ref, (n, seed, S, got["alpha"], a_ref)
    assert floors >= 2


def test_penalty_step_lambda_min_on_tensor_cores(ub):
    """The eigen-solver's matrix-vector products as the batched BF16 contraction (the iterate
    as two BF16 terms, FP32 accumulation; the perturbation on the diagonal only, so Q'_off
    is the integer Q_off): lambda_min and alpha against the oracle within 2e-3, as on the FP32
    path, for the states above the floor."""
    done = 0
    for n, seed, S in [(250, 1, 0), (250, 1, 5), (250, 0, 3), (600, 2, 0), (600, 2, 2)]:
        Q, b = I.random_ubqp(n, 0.1, seed)
        mu = np.diag(np.diag(I.perturbation(Q, seed)))
        Qp, bp, p, x = _state_at_outer_step(Q, b, mu, S)
        a_ref, m_ref, lam_ref, fb = O.penalty_step(Qp, bp, p, x)
        got = ub.penalty_probe(Qp, bp, p, x, precision=ub.BF16X2_TC)
        print(f"TC n={n} seed={seed} s={S}: oracle {lam_ref:.6e} gpu {got['lambda']:.6e} floor={fb}")
        assert got["n_active"] == m_ref
        if not fb:
            assert abs(got["lambda"] - lam_ref) <= 2e-3 * abs(lam_ref), (n, seed, S)
            assert abs(got["alpha"] - a_ref) <= 2e-3 * abs(a_ref), (n, seed, S)
            done += 1
    assert done >= 4


# ---- whole method (Alg. 3) -------------------------------------------------------------

def test_c1_solve_matches_oracle(ub):
    Q, b = I.c1_instance(50, 0)
    mu = I.perturbation(Q, 0)
    x, f, st = ub.solve(Q, b, mu=mu)
    assert f == O.objective(Q, b, x)                       # exact evaluation, bit for bit
    _, f_orc, st_orc = O.solve(Q, b, mu)
    assert f - f_orc <= 1e-3 * abs(f_orc)
    assert st["outer_steps"] >= 1 and st["inner_iters"] >= st["outer_steps"]


def test_bruteforce_optima_never_beaten(ub):
    cases = json.load(open(GOLD))["cases"]
    Qs, mus, fstar = [], [], []
    for c in cases:
        Q, b = I.random_ubqp(c["n"], 0.1, c["seed"])
        Qs.append(Q)
        mus.append(I.perturbation(Q, c["seed"]))
        fstar.append(c["f_star"])
    xs, obj, st = ub.solve_batched(Qs, None, mus)
    gaps = []
    for Q, x, f, fs in zip(Qs, xs, obj, fstar):
        assert f == O.objective(Q, None, x)
        assert f >= fs
        gaps.append(abs(f - fs) / abs(fs))
    assert np.mean(gaps) < 0.01 and sum(g == 0 for g in gaps) >= 14


def _oracle_objective_spread(Q, b, mu, k=3):
    """The oracle's objective on the input itself, with mu rounded to FP32, and under k
    symmetric 1e-7 relative changes of mu (FP32 rounding size)."""
    fs = [O.solve(Q, b, mu)[1], O.solve(Q, b, mu.astype(np.float32).astype(np.float64))[1]]
    for j in range(k):
        E = np.random.default_rng(j).standard_normal(Q.shape)
        fs.append(O.solve(Q, b, mu * (1 + 1e-7 * (E + E.T) / 2))[1])
    return fs


def test_maxcut_instances_fp32_exact_and_near_oracle(ub):
    """Max-Cut in 0/1 form (zero diagonal, +-1 weights, b = -W e; Sec. 5.3) on the FP32 path
    with the default symmetric storage: exact objective of the returned point and never below
    the exhaustive optimum at n = 18.  At n = 150 and 200 the bar is 0.1 % of the oracle where
    the oracle's own objective holds still under FP32-sized changes of its input; where it
    does not (the +-1 weights leave many near-equal local optima, and rounding picks one),
    the result must be no worse than the worst of those oracle runs, plus 0.1 %."""
    W, b = I.maxcut_ubqp(18, 0.5, 30)
    fstar, _ = enumerate_min(W, b)
    x, f, _ = ub.solve(W, b, mu=I.perturbation(W, 30))
    assert f == O.objective(W, b, x) and f >= fstar
    specs = [(150, 31), (200, 32), (170, 35), (190, 36)]
    data = [I.maxcut_ubqp(n, 0.3, s) for n, s in specs]
    mus = [I.perturbation(Wi, s) for (Wi, _), (n, s) in zip(data, specs)]
    xs, obj, st = ub.solve_batched([Wi for Wi, _ in data], [bi for _, bi in data], mus)
    assert st["storage"] in (1, 2)   # symmetric tiles or, at density 0.3, the sliced rows
    for (Wi, bi), mu, xi, fi in zip(data[:2], mus, xs, obj):
        assert fi == O.objective(Wi, bi, xi)
        fs = _oracle_objective_spread(Wi, bi, mu)
        print(f"maxcut n={Wi.shape[0]} gpu {fi} oracle {fs}")
        if max(fs) - min(fs) <= 1e-3 * abs(fs[0]):
            assert fi - fs[0] <= 1e-3 * abs(fs[0]), (fi, fs)
        else:
            assert fi - max(fs) <= 1e-3 * abs(max(fs)), (fi, fs)
    for (Wi, bi), xi, fi in zip(data[2:], xs[2:], obj[2:]):
        assert fi == O.objective(Wi, bi, xi)


@pytest.mark.parametrize("K", [5, 20])
def test_penalty_update_every_k_inner_iterations_vs_oracle(ub, K):
    """The paper's closing suggestion (Sec. 6) of updating the penalty in step with the inner
    iterations, read as ending each subproblem after K iterations of Alg. 2 (max_inner = K), so
    that p moves every K iterations.  Three C2-law instances (n = 250) on the default schedulers
    against the oracle with the same cap: exact objectives.  Subproblems cut short leave the
    run more sensitive to rounding (which local optimum it ends in), so the objective bar is
    0.1 % of the oracle where its own objective holds still under 16 FP32-rounding-sized
    changes of the stored entries (mu + 1e-7 Q E, E symmetric standard normal), else no worse
    than the worst of those oracle runs plus 0.1 %."""
    Qs, mus = [], []
    for seed in range(3):
        Q, _ = I.c2_instance(250, seed)
        Qs.append(Q)
        mus.append(I.perturbation(Q, seed))
    xs, obj, st = ub.solve_batched(Qs, None, mus, max_inner=K)
    po = O.opts(max_inner=K)
    for Q, mu, x, f in zip(Qs, mus, xs, obj):
        fs = [O.solve(Q, None, mu, o=po)[1]]
        for j in range(16):
            E = np.random.default_rng(j).standard_normal(Q.shape)
            fs.append(O.solve(Q, None, mu + 1e-7 * Q * (E + E.T) / 2, o=po)[1])
        print(f"max_inner={K}: gpu {f} oracle {fs[0]} spread {min(fs)} .. {max(fs)}")
        assert f == O.objective(Q, None, x)
        if max(fs) - min(fs) <= 1e-3 * abs(fs[0]):
            assert f - fs[0] <= 1e-3 * abs(fs[0]), (K, f, fs)
        else:
            assert f - max(fs) <= 1e-3 * abs(max(fs)), (K, f, fs)


def test_ragged_batch_matches_single_solves(ub):
    """Lanes of uneven size advance together without interfering: the batched call
    returns what separate calls return."""
    specs = [(37, 1), (120, 2), (64, 3), (250, 4)]
    Qs = [I.random_ubqp(n, 0.15, s)[0] for n, s in specs]
    mus = [I.perturbation(Q, s) for Q, (n, s) in zip(Qs, specs)]
    for kw in (dict(gemv_kernel=2, sym_storage=1, sparse_storage=2), dict(gemv_kernel=2, sym_storage=0, sparse_storage=2),
               dict(gemv_kernel=2, sparse_storage=1), dict(gemv_kernel=1, sparse_storage=2),
               dict(gemv_kernel=1, sparse_storage=1)):
        xs, obj, _ = ub.solve_batched(Qs, None, mus, **kw)
        for Q, mu, x, f in zip(Qs, mus, xs, obj):
            x1, f1, _ = ub.solve(Q, None, mu=mu, **kw)
            assert f1 == f and np.array_equal(x1, x), kw


@pytest.mark.parametrize("sparse", [2, 1])
@pytest.mark.parametrize("specs", [[(37, 1)], [(1000, 2)], [(2500, 3)], [(250, 4), (1000, 5), (61, 6)],
                                   [(300, 7), (2000, 8), (90, 9), (777, 10), (1500, 11)]])
def test_schedulers_agree_bitwise(ub, specs, sparse):
    """The lock-step scheduler (one launch per step of all lanes), the persistent lane loop
    (lanes advance independently inside one launch) and, for batches, the single-lane kernel
    with a group of CTAs per lane run the same row kernels in the same order of operations, so
    every solve is bit-identical: single lanes of 1, 63 and 157 row blocks and ragged batches
    of three and five sizes."""
    Qs = [I.random_ubqp(n, 0.1, s)[0] for n, s in specs]
    mus = [I.perturbation(Q, s) for Q, (n, s) in zip(Qs, specs)]
    kw = dict(max_outer=4, sym_storage=0, sparse_storage=sparse)   # dense rows, or sliced rows, in both
    x1, f1, s1 = ub.solve_batched(Qs, None, mus, gemv_kernel=1, **kw)
    x2, f2, s2 = ub.solve_batched(Qs, None, mus, gemv_kernel=2, **kw)
    assert s1["gemv_kernel"] == 1 and s2["gemv_kernel"] == 2
    assert np.array_equal(f1, f2) and all(np.array_equal(a, b) for a, b in zip(x1, x2))
    for key in ("inner_iters", "outer_steps", "lobpcg_iters", "jacobi_iters", "var_updates"):
        assert s1[key] == s2[key], key
    if len(specs) > 1:   # lane groups on the single-lane kernel (the same items as lock-step)
        x3, f3, s3 = ub.solve_batched(Qs, None, mus, gemv_kernel=3, **kw)
        assert s3["gemv_kernel"] == 3
        assert np.array_equal(f1, f3) and all(np.array_equal(a, b) for a, b in zip(x1, x3))
        for key in ("inner_iters", "outer_steps", "lobpcg_iters", "jacobi_iters", "var_updates"):
            assert s1[key] == s3[key], key
    _, _, s0 = ub.solve_batched(Qs, None, mus, max_outer=4)
    # the default at density 0.1: the sliced rows (their bytes are fewer than the symmetric
    # tiles'), and on them the single-lane kernel with a group of CTAs per lane
    assert s0["gemv_kernel"] == 3
    assert s0["storage"] == 2


@pytest.mark.parametrize("n,seed,budget", [(37, 1, 0), (50, 0, 0), (256, 2, 0), (300, 3, 0), (1000, 4, 0),
                                           (2500, 5, 0), (1000, 6, 3)])
def test_single_lane_kernel_agrees_with_lockstep_bitwise(ub, n, seed, budget):
    """The single-lane persistent kernel (two grid barriers per step, every CTA taking the same
    decision) computes exactly what the lock-step scheduler computes with the same rows per
    item: same objective, same point, same step counts.  One CTA for n <= 256, many for larger n,
    and relaunches every 3 steps."""
    Q, _ = I.random_ubqp(n, 0.1, seed)
    mu = I.perturbation(Q, seed)
    kw = dict(max_outer=6, rows_per_item=16, sparse_storage=2)
    if budget == 0 and n in (1000, 2500):   # the sliced rows too, with the same items in both
        for rb in (64, 32):   # 32: one slice per CTA, the warp-level epilogue
            kw2 = dict(max_outer=6, rows_per_item=rb, sparse_storage=1)
            x1, f1, s1 = ub.solve(Q, None, mu=mu, gemv_kernel=1, **kw2)
            x3, f3, s3 = ub.solve(Q, None, mu=mu, gemv_kernel=3, **kw2)
            assert s1["storage"] == 2 and s3["storage"] == 2
            assert f1 == f3 and np.array_equal(x1, x3) and s1["inner_iters"] == s3["inner_iters"]
    x1, f1, s1 = ub.solve(Q, None, mu=mu, gemv_kernel=1, **kw)
    x3, f3, s3 = ub.solve(Q, None, mu=mu, gemv_kernel=3, lane_budget=budget, **kw)
    assert s1["gemv_kernel"] == 1 and s3["gemv_kernel"] == 3
    assert f1 == f3 and np.array_equal(x1, x3)
    for key in ("inner_iters", "inner_steps", "outer_steps", "lobpcg_iters", "jacobi_iters", "var_updates"):
        assert s1[key] == s3[key], key
    if budget:
        assert s3["kernel_launches"] > 100


@pytest.mark.parametrize("case", ["mixed", "mixed_budget", "many", "large"])
def test_lane_groups_agree_with_lockstep_bitwise(ub, case):
    """Several lanes on the single-lane kernel.  "mixed": every lane on its own group of CTAs
    (sliced rows, 32-row items, a CTA computing up to five slices per step), also relaunched
    every 7 steps; "many": more lanes than resident CTAs, so one-CTA groups run several lanes in
    turn (lanes of one slice keep Alg. 2 in shared memory); "large": n = 6000 next to smaller
    lanes.  Same objectives, points and step counts as the lock-step scheduler with the same
    items."""
    if case.startswith("mixed"):
        specs = [(2500, 11), (1000, 12), (500, 13), (250, 14), (37, 15), (1000, 16), (300, 17)]
    elif case == "large":   # two vectors of 6016 floats per CTA in shared memory
        specs = [(6000, 21), (1500, 22), (300, 23)]
    else:
        specs = [(20 + (i % 5) * 7, 100 + i) for i in range(400)]
    Qs = [I.random_ubqp(n, 0.1, s)[0] for n, s in specs]
    mus = [I.perturbation(Q, s) for Q, (n, s) in zip(Qs, specs)]
    kw = dict(max_outer=3 if case == "large" else 4, rows_per_item=32, sparse_storage=1)
    budget = {"mixed": 0, "mixed_budget": 7, "many": 5, "large": 0}[case]
    x1, f1, s1 = ub.solve_batched(Qs, None, mus, gemv_kernel=1, **kw)
    x3, f3, s3 = ub.solve_batched(Qs, None, mus, gemv_kernel=3, lane_budget=budget, **kw)
    assert s1["gemv_kernel"] == 1 and s3["gemv_kernel"] == 3 and s3["storage"] == 2
    assert np.array_equal(f1, f3) and all(np.array_equal(a, b) for a, b in zip(x1, x3))
    for key in ("inner_iters", "inner_steps", "outer_steps", "lobpcg_iters", "jacobi_iters", "var_updates"):
        assert s1[key] == s3[key], key
    if case == "mixed":   # the automatic choice for FP32 lanes on the sliced storage
        _, _, s0 = ub.solve_batched(Qs, None, mus, max_outer=1)
        assert s0["gemv_kernel"] == 3 and s0["storage"] == 2


def test_lane_loop_small_budget_relaunches(ub):
    """A budget of 3 steps per launch makes the host relaunch the loop hundreds of times;
    lanes that finish early stay in the seeded ring as skip entries.  Same bits as one
    long launch, and the step count is the busiest lane's."""
    specs = [(300, 7), (64, 8), (129, 9)]
    Qs = [I.random_ubqp(n, 0.1, s)[0] for n, s in specs]
    mus = [I.perturbation(Q, s) for Q, (n, s) in zip(Qs, specs)]
    x1, f1, s1 = ub.solve_batched(Qs, None, mus, gemv_kernel=2)
    x2, f2, s2 = ub.solve_batched(Qs, None, mus, gemv_kernel=2, lane_budget=3)
    assert np.array_equal(f1, f2) and all(np.array_equal(a, b) for a, b in zip(x1, x2))
    assert s1["ticks"] == s2["ticks"] and s2["kernel_launches"] > s1["kernel_launches"] + 100
    _, _, s3 = ub.solve_batched(Qs, None, mus, profile_kernels=2, max_outer=2)
    assert s3["gemv_kernel"] == 1                       # the per-step timeline runs lock-step


def test_sym_lanes_of_every_block_count_reseeded(ub):
    """Symmetric storage, lanes of 1 to 9 row blocks: relaunching the loop every 3 steps seeds
    lanes in tile steps and in evaluation steps (row blocks only) again and again.  Same bits
    as one long launch and as a lane solved alone."""
    ns = [100, 200, 300, 450, 600, 700, 850, 1000, 1100]
    Qs = [I.random_ubqp(n, 0.1, 20 + i)[0] for i, n in enumerate(ns)]
    mus = [I.perturbation(Q, 20 + i) for i, Q in enumerate(Qs)]
    kw = dict(gemv_kernel=2, sym_storage=1, sparse_storage=2, max_outer=4)
    x1, f1, s1 = ub.solve_batched(Qs, None, mus, **kw)
    x2, f2, s2 = ub.solve_batched(Qs, None, mus, lane_budget=3, **kw)
    assert s1["sym_storage"] == 1 and s2["sym_storage"] == 1
    assert np.array_equal(f1, f2) and all(np.array_equal(a, b) for a, b in zip(x1, x2))
    assert s1["ticks"] == s2["ticks"] and s2["kernel_launches"] > s1["kernel_launches"] + 100
    x3, f3, _ = ub.solve(Qs[4], None, mu=mus[4], **kw)   # the 5-block lane alone
    assert f3 == f1[4] and np.array_equal(x3, x1[4])


def test_restarts_keep_best_and_are_exact(ub):
    Q, b = I.random_ubqp(80, 0.2, 9, b_range=(-20, 20))
    mu = I.perturbation(Q, 9)
    starts = I.random_starts(80, 7, 9)
    x1, f1, _ = ub.solve(Q, b, mu=mu, gemv_kernel=2)   # start 0 alone, in the batch's mode
    x8, f8, st = ub.solve(Q, b, mu=mu, starts=starts, restarts=8, gemv_kernel=2)
    assert st["lanes"] == 8
    assert f8 <= f1 and f8 == O.objective(Q, b, x8)
    for r in range(7):   # each start alone, through the oracle, is never better than the batch
        _, fr, _ = O.solve(Q, b, mu, x_start=starts[r])
        assert f8 <= fr + 1e-3 * abs(fr)


@pytest.mark.parametrize("sched", ["dense", "sym", "sliced"])
def test_full_size_c2_instance_properties(ub, sched):
    """n = 2500 (largest single-instance size; 210 symmetric tiles): exact objective of the
    returned point, binary output and a finished run."""
    Q, _ = I.c2_instance(2500, 0)
    x, f, st = ub.solve(Q, None, mu=I.perturbation(Q, 0), **SCHEDULES[sched])
    assert set(np.unique(x)) <= {0, 1}
    assert f == O.objective(Q, None, x)
    assert st["status"] == 0 and st["lanes_capped"] == 0


# ---- edge cases ------------------------------------------------------------------------

def test_tiny_and_degenerate_instances(ub):
    x, f, _ = ub.solve(np.array([[3.0]]), np.array([-5.0]))
    assert f == -2.0 and x.tolist() == [1]
    x, f, _ = ub.solve(np.array([[3.0]]), np.array([5.0]))
    assert f == 0.0 and x.tolist() == [0]
    Q = np.array([[1.0, -4.0], [-4.0, 1.0]])
    x, f, _ = ub.solve(Q, np.zeros(2))
    assert f == O.objective(Q, np.zeros(2), x) and f == -6.0
    x, f, _ = ub.solve(np.zeros((5, 5)))           # f = 0 everywhere
    assert f == 0.0


def test_lane_loop_wait_limit_runs_out_and_the_device_stays_usable(ub):
    """Failure detection without a GPU fault: with the ring-slot wait of the lane loop limited
    to 1 us, CTAs that find no entry ready give up, set the error flag and leave (no copy is
    in flight during that wait), the others leave at their own next wait, and the call
    returns UBQP_ETIMEOUT with the limit in ubqp_last_error().  The same context then solves a
    fresh batch with the default limit, exactly."""
    specs = [(500, 1), (300, 2), (700, 3), (250, 4), (600, 5), (450, 6)]
    Qs = [I.random_ubqp(n, 0.1, s)[0] for n, s in specs]
    mus = [I.perturbation(Q, s) for Q, (n, s) in zip(Qs, specs)]
    with pytest.raises(ub.UBQPError) as e:
        ub.solve_batched(Qs, None, mus, gemv_kernel=2, wait_limit_us=1)
    assert e.value.status == -6
    assert "bounded wait in the lane loop ran out" in str(e.value) and "limit 1 us" in str(e.value)
    xs, obj, st = ub.solve_batched(Qs, None, mus, gemv_kernel=2)
    assert st["gemv_kernel"] == 2
    for Q, x, f in zip(Qs, xs, obj):
        assert f == O.objective(Q, None, x)
    x1, f1, _ = ub.solve(Qs[0], None, mu=mus[0], gemv_kernel=2)
    assert f1 == obj[0] and np.array_equal(x1, xs[0])
    # the single-lane kernel's grid barrier wait, the same way
    Q, _ = I.random_ubqp(2500, 0.1, 9)
    with pytest.raises(ub.UBQPError) as e:
        ub.solve(Q, None, mu=I.perturbation(Q, 9), wait_limit_us=1)
    assert e.value.status == -6 and "single-lane kernel" in str(e.value)
    x, f, st = ub.solve(Q, None, mu=I.perturbation(Q, 9), max_outer=3)
    assert st["gemv_kernel"] == 3 and f == O.objective(Q, None, x)


def test_errors_are_reported(ub):
    Q = np.array([[0.0, 1.0], [2.0, 0.0]])
    with pytest.raises(ub.UBQPError) as e:
        ub.solve(Q)
    assert e.value.status == -2
    Q = np.array([[0.0, np.nan], [np.nan, 0.0]])
    with pytest.raises(ub.UBQPError) as e:
        ub.solve(Q)
    assert e.value.status == -3
    with pytest.raises(ub.UBQPError) as e:
        ub.solve(np.eye(3), eta=1.5)
    assert e.value.status == -1
    x, f, _ = ub.solve(np.eye(3) * -1.0)            # the device is still usable
    assert f == -3.0


# ---- penalized objective and its gradient (autograd) -------------------------------------

def _c3_case(dtype, with_p):
    """C3 inputs as the GPU holds them: Q, b integers (exact in both dtypes), p and the 64 box
    points rounded to the tested dtype, so that the oracle evaluates the same numbers."""
    Q, b = I.c3_instance(1000, 1)
    X = I.box_points(1000, 64, 1)
    p = np.random.default_rng(1).uniform(0, 100, 1000) if with_p else np.zeros(1000)
    if dtype == "float32":
        X, p = _r32(X), _r32(p)
    return Q, b, p, X


@pytest.mark.parametrize("with_p", [False, True])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_penalized_eval_all_points_vs_oracle(ub, dtype, with_p):
    """h and grad h of problem (p) (Sec. 4.1) through PenalizedObjective (forward:
    ubqp_penalized_eval on the inner loop's GEMV kernel; backward: ubqp_penalized_vjp) on all
    64 C3 points, against the FP64 oracle on the same inputs.  Bar: 1e-5 (FP32) / 1e-12 (FP64)
    relative, h to max(|h|, 1) and g to max_i |g_i| of each point."""
    import torch
    Q, b, p, X = _c3_case(dtype, with_p)
    dt = getattr(torch, dtype)
    Qt, bt, pt = (torch.tensor(a, dtype=dt, device="cuda") for a in (Q, b, p))
    Xt = torch.tensor(X, dtype=dt, device="cuda", requires_grad=True)
    h = ub.PenalizedObjective.apply(Xt, Qt, bt, pt)
    h.sum().backward()
    G = Xt.grad.double().cpu().numpy()
    H = h.detach().double().cpu().numpy()
    tol = 1e-5 if dtype == "float32" else 1e-12
    worst_h = worst_g = 0.0
    for r in range(64):
        h_ref, g_ref = O.penalized(Q, b, p, X[r])
        worst_h = max(worst_h, abs(H[r] - h_ref) / max(abs(h_ref), 1.0))
        worst_g = max(worst_g, np.max(np.abs(G[r] - g_ref)) / np.max(np.abs(g_ref)))
    print(f"penalized {dtype} p={'U[0,100]' if with_p else 0}: worst rel h {worst_h:.2e}, g {worst_g:.2e}")
    assert worst_h <= tol and worst_g <= tol, (worst_h, worst_g)


def test_penalized_backward_vs_central_differences_of_the_gpu_forward(ub):
    """The hand-written backward against central differences (h = 1e-3, FP64) of the GPU
    forward itself, for x, p and b.  h is quadratic in x and linear in p and b, so central
    differences are exact up to rounding of the forward values (about 1e-11 of h here): bar
    1e-8 relative to the largest gradient entry."""
    import torch
    Q, b, p, X = _c3_case("float64", True)
    X = X[:4]
    w = np.array([1.0, -0.5, 2.0, 0.25])          # grad_out of h: a weighted sum of the 4 points
    Qt = torch.tensor(Q, dtype=torch.float64, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True)
    pt = torch.tensor(p, dtype=torch.float64, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    (ub.PenalizedObjective.apply(Xt, Qt, bt, pt) * wt).sum().backward()
    gx, gb, gp = (t.grad.cpu().numpy() for t in (Xt, bt, pt))

    def F(Xv, bv, pv):
        h, _ = ub.penalized_eval(Qt, torch.tensor(bv, dtype=torch.float64, device="cuda"),
                                 torch.tensor(pv, dtype=torch.float64, device="cuda"),
                                 torch.tensor(Xv, dtype=torch.float64, device="cuda"), want_g=False)
        return float((h.cpu().numpy() * w).sum())

    e = 1e-3
    idx = [0, 1, 17, 123, 500, 998, 999]
    for r in (0, 2):
        for i in idx:
            Xp, Xm = X.copy(), X.copy()
            Xp[r, i] += e
            Xm[r, i] -= e
            fd = (F(Xp, b, p) - F(Xm, b, p)) / (2 * e)
            assert abs(fd - gx[r, i]) <= 1e-8 * np.max(np.abs(gx[r])), (r, i, fd, gx[r, i])
    for i in idx:
        bp_, bm_ = b.copy(), b.copy()
        bp_[i] += e
        bm_[i] -= e
        assert abs((F(X, bp_, p) - F(X, bm_, p)) / (2 * e) - gb[i]) <= 1e-8 * np.max(np.abs(gb))
        pp_, pm_ = p.copy(), p.copy()
        pp_[i] += e
        pm_[i] -= e
        assert abs((F(X, b, pp_) - F(X, b, pm_)) / (2 * e) - gp[i]) <= 1e-8 * np.max(np.abs(gp))
    # and against the oracle's gradient of each point, weighted
    for r in range(4):
        _, g_ref = O.penalized(Q, b, p, X[r])
        assert np.max(np.abs(gx[r] - w[r] * g_ref)) <= 1e-12 * np.max(np.abs(w[r] * g_ref))


@pytest.mark.parametrize("n", [1, 3, 37, 1001, 4099])
def test_penalized_eval_unpadded_rows_of_any_length(ub, n):
    """Rows of the caller's Q start at any 4-byte offset when n is not a multiple of 4: the
    row dot takes the entries before the first 16-byte boundary and after the last whole group
    one by one.  FP32 and FP64 against the oracle, at sizes 1, 3, 37, 1001 and 4099."""
    import torch
    rng = np.random.default_rng(n)
    Q = rng.integers(-100, 101, (n, n)).astype(np.float64)
    Q = np.triu(Q) + np.triu(Q, 1).T
    b = rng.integers(-50, 51, n).astype(np.float64)
    p = rng.uniform(0, 100, n)
    X = rng.random((5, n))
    for dtype, tol in (("float32", 1e-5), ("float64", 1e-12)):
        Xd, pd = (_r32(X), _r32(p)) if dtype == "float32" else (X, p)
        dt = getattr(torch, dtype)
        h, g = ub.penalized_eval(*(torch.tensor(a, dtype=dt, device="cuda") for a in (Q, b, pd, Xd)))
        H, G = h.double().cpu().numpy(), g.double().cpu().numpy()
        for r in range(5):
            h_ref, g_ref = O.penalized(Q, b, pd, Xd[r])
            assert abs(H[r] - h_ref) <= tol * max(abs(h_ref), 1.0), (dtype, r)
            assert np.max(np.abs(G[r] - g_ref)) <= tol * max(np.max(np.abs(g_ref)), 1.0), (dtype, r)
