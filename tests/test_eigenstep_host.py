"""Host pins of the solver's 3 x 3 eigen-step (the Rayleigh-Ritz step of the LOBPCG iteration
for lambda_min in Lemma 3.1, and the Jacobi eigen-solver it calls), run through their host
form (tests/eigenstep_harness.cu, built here with nvcc) against numpy / scipy:

- small_sym_eig_min: the smallest eigenvalue and a unit eigenvector of k x k symmetric
  matrices, k = 1, 2, 3, with the entries outside k x k ignored;
- rayleigh_ritz: the smallest eigenpair of the pencil (A_g, B_g) of Gram matrices of
  span{x, w, p} (or {x, w}), its vector B_g-normalized; a nearly dependent p is dropped (the
  result is the {x, w} one, bit for bit); a zero x or w is a breakdown.

The device runs the same code with the hardware reciprocal square root; these checks hold
the logic (masking, rotations, Cholesky, back-transformation, breakdown rules)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("eigenstep") / "eigenstep_harness")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "eigenstep_harness.cu"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.strip().splitlines()
    return run


def _f32(v):
    return float(np.float32(v))


def _eig_line(k, M):
    return "eig %d " % k + " ".join("%.9g" % _f32(M[i, j]) for i, j in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)))


def test_small_sym_eig_min_against_eigvalsh(harness):
    rng = np.random.default_rng(11)
    Ms = []
    for _ in range(200):
        A = rng.normal(size=(3, 3))
        Ms.append((A + A.T) / 2)
    out = harness([_eig_line(3, M) for M in Ms])
    for M, line in zip(Ms, out):
        M = M.astype(np.float32).astype(np.float64)
        lam, *v = map(float, line.split())
        v = np.array(v)
        w = np.linalg.eigvalsh(M)
        scale = np.abs(w).max()
        assert abs(lam - w[0]) <= 2e-6 * scale, (lam, w)
        assert abs(np.linalg.norm(v) - 1.0) <= 1e-5
        assert np.linalg.norm(M @ v - lam * v) <= 2e-5 * scale


def test_small_sym_eig_min_ignores_entries_outside_k(harness):
    rng = np.random.default_rng(12)
    lines, blocks = [], []
    for k in (1, 2):
        for _ in range(50):
            A = rng.normal(size=(3, 3))
            M = (A + A.T) / 2
            M[k:, :] = M[:, k:] = 1e3 * rng.normal()   # garbage outside the k x k block
            M[k:, :k] = M[:k, k:].T
            lines.append(_eig_line(k, M))
            blocks.append((k, M))
    for (k, M), line in zip(blocks, harness(lines)):
        lam, *v = map(float, line.split())
        B = M.astype(np.float32).astype(np.float64)[:k, :k]
        w = np.linalg.eigvalsh(B)
        assert abs(lam - w[0]) <= 2e-6 * np.abs(w).max()
        assert all(x == 0.0 for x in v[k:])
        if k == 1:
            assert v[0] == 1.0


def _gram(A, vecs):
    V = np.stack(vecs, axis=1)
    return V.T @ A @ V, V.T @ V


def _rr_line(has_p, Ag, Bg):
    idx = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    ga = [Ag[i, j] if max(i, j) < Ag.shape[0] else 0.0 for i, j in idx]
    gb = [Bg[i, j] if max(i, j) < Bg.shape[0] else 0.0 for i, j in idx]
    return "rr %d " % has_p + " ".join("%.9g" % _f32(t) for t in ga + gb)


def _pencil_min(Ag, Bg):
    from scipy.linalg import eigh
    return eigh(Ag, Bg, eigvals_only=True)[0]


@pytest.mark.parametrize("has_p", [1, 0])
def test_rayleigh_ritz_smallest_pair_of_the_gram_pencil(harness, has_p):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(13 + has_p)
    cases = []
    for _ in range(100):
        n = 40
        A = rng.normal(size=(n, n))
        A = (A + A.T) / 2
        vecs = [rng.normal(size=n) for _ in range(3 if has_p else 2)]
        Ag, Bg = _gram(A, vecs)
        cases.append((Ag, Bg))
    out = harness([_rr_line(has_p, Ag, Bg) for Ag, Bg in cases])
    for (Ag, Bg), line in zip(cases, out):
        tok = line.split()
        assert tok[0] == "ok", line
        lam = float(tok[1])
        k = 3 if has_p else 2
        c = np.array(list(map(float, tok[2:2 + k])))
        assert all(float(t) == 0.0 for t in tok[2 + k:])
        Ag32, Bg32 = (M.astype(np.float32).astype(np.float64) for M in (Ag, Bg))
        ref = _pencil_min(Ag32, Bg32)
        scale = np.abs(Ag32).max()
        assert abs(lam - ref) <= 1e-4 * scale, (lam, ref)
        assert abs(c @ Bg32 @ c - 1.0) <= 1e-3
        assert np.linalg.norm(Ag32 @ c - lam * (Bg32 @ c)) <= 1e-3 * scale * np.linalg.norm(c)


def test_rayleigh_ritz_drops_a_dependent_direction_and_reports_breakdown(harness):
    rng = np.random.default_rng(14)
    n = 40
    A = rng.normal(size=(n, n))
    A = (A + A.T) / 2
    x, w = rng.normal(size=n), rng.normal(size=n)
    p = x + 1e-2 * rng.normal(size=n)            # nearly dependent on x: Cholesky pivot ~1e-4 < 1e-3
    Ag3, Bg3 = _gram(A, [x, w, p])
    Ag2, Bg2 = _gram(A, [x, w])
    zero_w = _gram(A, [x, np.zeros(n), p])
    lines = [_rr_line(1, Ag3, Bg3), _rr_line(0, Ag2, Bg2),
             _rr_line(1, *zero_w),                                   # w = 0: no basis left
             _rr_line(0, *_gram(A, [np.zeros(n), w]))]               # x = 0
    dep, plain, brk_w, brk_x = harness(lines)
    assert dep == plain and dep.startswith("ok"), (dep, plain)
    assert brk_w == "fail" and brk_x == "fail"
