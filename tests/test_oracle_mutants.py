"""The oracle's pins catch plausible mistakes (CPU).

Each case plants one mistake in a copy of the oracle's C source (a dropped term, a flipped
sign, a swapped operand, a wrong factor), compiles the copy with gcc into a temporary
directory, and runs every pin of ``tests/test_oracle.py`` against it in a child process: at
least one pin must fail.  The unmodified source, built the same way, must pass them all.
The oracle under ``oracle/`` itself is never modified.
"""
import importlib.util
import os
import pathlib
import subprocess
import sys

import pytest

HERE = pathlib.Path(__file__).resolve().parent
ROOT = HERE.parent
SRC = ROOT / "oracle" / "ubqp_oracle.c"

# (name, exact text in the oracle source, replacement)
MUTANTS = [
    ("objective drops b", "if (b) f += b[i];", ";"),
    ("objective uses Q_ji of unset j", "if (x[j]) row += Q[IDX(i, j, n)];", "row += Q[IDX(i, j, n)];"),
    ("gamma without the factor 2", "gamma[i] = 2.0 * r + fabs(bi) + margin;", "gamma[i] = r + fabs(bi) + margin;"),
    ("b' = b + gamma", "bp[i] = bi - gamma[i];", "bp[i] = bi + gamma[i];"),
    ("gamma left off the diagonal", "Qp[IDX(i, i, n)] += gamma[i];", ";"),
    ("x0 solves 2Q'x = b'", "double t = -bp[i];", "double t = bp[i];"),
    ("x0 off-diagonal factor", "double t = 2.0 * Qp[IDX(i, j, n)];", "double t = Qp[IDX(i, j, n)];"),
    ("h penalty sign", "pi * (x[i] - x[i] * x[i]);", "pi * (x[i] + x[i] * x[i]);"),
    ("gradient penalty factor", "if (g) g[i] = 2.0 * qx - 2.0 * pi * x[i] + bi + pi;",
     "if (g) g[i] = 2.0 * qx - pi * x[i] + bi + pi;"),
    ("gradient drops p", "if (g) g[i] = 2.0 * qx - 2.0 * pi * x[i] + bi + pi;",
     "if (g) g[i] = 2.0 * qx - 2.0 * pi * x[i] + bi;"),
    ("KKT: J side sign", "else if (x[i] <= 0.0) v = g[i] < 0.0 ? -g[i] : 0.0;",
     "else if (x[i] <= 0.0) v = g[i] > 0.0 ? g[i] : 0.0;"),
    ("KKT: interior ignored", "if (x[i] > 0.0 && x[i] < 1.0) v = fabs(g[i]);", "if (x[i] > 0.0 && x[i] < 1.0) v = 0.0;"),
    ("rho: P* added", "double q = Q[IDX(i, j, n)] - (i == j && p ? p[i] : 0.0);",
     "double q = Q[IDX(i, j, n)] + (i == j && p ? p[i] : 0.0);"),
    ("rho: b + p without p", "double bb = (b ? b[i] : 0.0) + (p ? p[i] : 0.0);", "double bb = (b ? b[i] : 0.0);"),
    ("Householder update factor", "double K = 0.5 * beta * pv;", "double K = beta * pv;"),
    ("Sturm recurrence sign", "q = (a[i] - x) - e[i - 1] * e[i - 1] / q;", "q = (a[i] - x) + e[i - 1] * e[i - 1] / q;"),
    ("penalty step: Z^(1/2) for Z^(-1/2)", "rz[m] = 1.0 / sqrt(z);", "rz[m] = sqrt(z);"),
    ("penalty step: Q' + P*", "double q = Qp[IDX(i, j, n)] - (i == j ? p[i] : 0.0);",
     "double q = Qp[IDX(i, j, n)] + (i == j ? p[i] : 0.0);"),
    ("penalty step without eta", "if (lam > floor) alpha = o->eta * lam;", "if (lam > floor) alpha = lam;"),
    ("penalty floor never doubles", "ldexp(floor, consecutive < 60 ? consecutive : 60)", "floor"),
    ("inner gradient drops -2 p x", "g[i] = 2.0 * qx - 2.0 * p[i] * x[i] + bp[i] + p[i];",
     "g[i] = 2.0 * qx + bp[i] + p[i];"),
    ("BB steps swapped", "double a = (k % 2 == 1) ? ss / sy : sy / yy;", "double a = (k % 2 == 1) ? sy / yy : ss / sy;"),
    ("BB1 inverted", "double a = (k % 2 == 1) ? ss / sy : sy / yy;", "double a = (k % 2 == 1) ? sy / ss : sy / yy;"),
    ("no projection", "x[i] = clip01(x[i] - alpha * g[i]);", "x[i] = x[i] - alpha * g[i];"),
    ("first step from the 1-norm of Q' alone", "r += fabs(Qp[IDX(i, j, n)] - (i == j ? p[i] : 0.0));",
     "r += fabs(Qp[IDX(i, j, n)]);"),
    ("PPA step without the 2", "double xn = clip01(x[i] - g[i] / (2.0 * hp[i]));",
     "double xn = clip01(x[i] - g[i] / hp[i]);"),
    ("PPA h_p + p", "for (int i = 0; i < n; ++i) hp[i] = fmax(hp[i] - p[i], eps);",
     "for (int i = 0; i < n; ++i) hp[i] = fmax(hp[i] + p[i], eps);"),
    ("Cholesky diagonal sign", "for (int k = 0; k < j; ++k) s -= L[IDX(j, k, n)] * L[IDX(j, k, n)];",
     "for (int k = 0; k < j; ++k) s += L[IDX(j, k, n)] * L[IDX(j, k, n)];"),
    ("back substitution with L for L^T", "for (int k = i + 1; k < n; ++k) t -= L[IDX(k, i, n)] * x0[k];",
     "for (int k = i + 1; k < n; ++k) t -= L[IDX(i, k, n)] * x0[k];"),
    ("perturbation ignored", "Qp[t] = Q[t] + (mu ? mu[t] : 0.0);", "Qp[t] = Q[t];"),
    ("BB keeps steps of negative curvature", "if (!(sy > 0.0) || !isfinite(a)) a = alpha;",
     "if (!isfinite(a)) a = alpha;"),
    ("absolute KKT test", "if (orc_kkt_residual(n, x, g) / rho < o->tol_inner)", "if (orc_kkt_residual(n, x, g) < o->tol_inner)"),
    ("best point not stored", "memcpy(x_best, xr, (size_t)n);", ";"),
    ("outer test on the rounded point", "if (binarity(n, x) <= o->tol_outer)", "if (binarity(n, x) <= 0.5)"),
    ("rounding flipped", "for (int i = 0; i < n; ++i) xr[i] = x[i] > 0.5;", "for (int i = 0; i < n; ++i) xr[i] = x[i] < 0.5;"),
    ("keeps the worst point", "if (f < best) {", "if (f > best || best == INFINITY) {"),
    ("penalty update without z", "for (int i = 0; i < n; ++i) p[i] += alpha * (x[i] - x[i] * x[i]);",
     "for (int i = 0; i < n; ++i) p[i] += alpha;"),
    ("penalty update sign", "for (int i = 0; i < n; ++i) p[i] += alpha * (x[i] - x[i] * x[i]);",
     "for (int i = 0; i < n; ++i) p[i] -= alpha * (x[i] - x[i] * x[i]);"),
]


def _compile(text: str, out: pathlib.Path) -> pathlib.Path:
    c = out.with_suffix(".c")
    c.write_text(text)
    so = out.with_suffix(".so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-I", str(SRC.parent), "-o", str(so), str(c), "-lm"],
                   check=True)
    return so


def _pins():
    """Every test of tests/test_oracle.py as a zero-argument call (parametrized ones expanded)."""
    spec = importlib.util.spec_from_file_location("oracle_pins", HERE / "test_oracle.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    calls = []
    for name in sorted(n for n in dir(mod) if n.startswith("test_")):
        fn = getattr(mod, name)
        params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if not params:
            calls.append((name, fn, {}))
            continue
        assert len(params) == 1
        argnames, values = params[0].args[:2]
        argnames = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
        for v in values:
            v = v if len(argnames) > 1 else (v,)
            calls.append((f"{name}{list(v)}", fn, dict(zip(argnames, v))))
    return calls


def run_pins(so_path: str) -> int:
    """Child process: point the oracle wrapper at ``so_path`` and run every pin; print the
    failing ones and return how many failed."""
    import oracle as O
    O._lib = O.load(so_path)
    failed = 0
    for name, fn, kw in _pins():
        try:
            fn(**kw)
        except Exception as e:   # an assertion, or an error the mistake provokes
            failed += 1
            print(f"FAIL {name}: {type(e).__name__}", flush=True)
    return failed


def _child(so: pathlib.Path):
    code = ("import sys; sys.path[:0] = [sys.argv[2], sys.argv[3]]; import test_oracle_mutants as m; "
            "sys.exit(min(m.run_pins(sys.argv[1]), 100))")
    return subprocess.run([sys.executable, "-c", code, str(so), str(HERE), str(ROOT)], capture_output=True,
                          text=True, timeout=300, cwd=str(ROOT), env=dict(os.environ, OMP_NUM_THREADS="1"))


def test_unmodified_copy_passes_every_pin(tmp_path):
    so = _compile(SRC.read_text(), tmp_path / "clean")
    r = _child(so)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    text = SRC.read_text()
    assert text.count(old) == 1, f"pattern of '{name}' not unique in the oracle source"
    so = _compile(text.replace(old, new), tmp_path / "mutant")
    r = _child(so)
    assert r.returncode != 0, f"'{name}' survived every pin\n{r.stdout}{r.stderr}"
