/*
 * FP64 CPU oracle of the vectorized PSDP method (arXiv 2408.04875).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark.  Never part of the product path.
 *
 * Every function follows one passage of the paper, cited in its comment, written
 * as plain loops in double precision.  See ubqp_oracle.h for the readings of the
 * points the paper leaves open.
 */
#include "ubqp_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, n) ((size_t)(i) * (size_t)(n) + (size_t)(j))

void orc_opts_default(orc_opts* o)
{
    o->method = 0;
    o->max_outer = 1000;       /* Sec. 5, PABB/PPA settings */
    o->max_inner = 10000;
    o->tol_inner = 1e-5;       /* Eq. (cret) delta */
    o->tol_outer = 1e-5;       /* Alg. 3 while-test */
    o->eta = 0.9;              /* Eq. (eq:alpha1): value not given, 0 < eta < 1 */
    o->gamma_margin = 1.0;     /* Eq. (gamma): strict ">" */
    o->alpha_min = 1e-10;
    o->alpha_max = 1e10;
    o->tau_z = 1e-12;
    o->eps_hp_rel = 1e-8;      /* Sec. 3.1: "arbitrarily small" epsilon */
    o->lambda_floor_rel = 4.0;
    o->fp32_noise = 0.0;       /* rounding model off */
    o->noise_seed = 0;
}

/* Eq. (bqp): f(x) = x^T Q x + b^T x on a binary point. */
double orc_objective(int n, const double* Q, const double* b, const uint8_t* x)
{
    double f = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!x[i]) continue;
        double row = 0.0;
        for (int j = 0; j < n; ++j)
            if (x[j]) row += Q[IDX(i, j, n)];
        f += row;
        if (b) f += b[i];
    }
    return f;
}

/* Sec. 3.5 (reformulation) after the symmetric perturbation of Sec. 3.5 (random
 * perturbation): Q' = Q + mu + Diag(gamma), b' = b - gamma, gamma from Eq. (gamma). */
void orc_reformulate(int n, const double* Q, const double* b, const double* mu, double margin,
                     double* Qp, double* bp, double* gamma)
{
    for (size_t t = 0; t < (size_t)n * n; ++t) Qp[t] = Q[t] + (mu ? mu[t] : 0.0);
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += fabs(Qp[IDX(i, j, n)]);
        double bi = b ? b[i] : 0.0;
        gamma[i] = 2.0 * r + fabs(bi) + margin;
        Qp[IDX(i, i, n)] += gamma[i];
        bp[i] = bi - gamma[i];
    }
}

/* Eq. (gamma): first-order condition 2 Q' x = gamma - b = -b', solved by Cholesky. */
int orc_initial_point(int n, const double* Qp, const double* bp, double* x0)
{
    double* L = (double*)calloc((size_t)n * n, sizeof(double));
    double* y = (double*)malloc((size_t)n * sizeof(double));
    if (!L || !y) { free(L); free(y); return -2; }
    for (int j = 0; j < n; ++j) {
        double s = 2.0 * Qp[IDX(j, j, n)];
        for (int k = 0; k < j; ++k) s -= L[IDX(j, k, n)] * L[IDX(j, k, n)];
        if (!(s > 0.0)) { free(L); free(y); return -1; }
        double ljj = sqrt(s);
        L[IDX(j, j, n)] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = 2.0 * Qp[IDX(i, j, n)];
            for (int k = 0; k < j; ++k) t -= L[IDX(i, k, n)] * L[IDX(j, k, n)];
            L[IDX(i, j, n)] = t / ljj;
        }
    }
    for (int i = 0; i < n; ++i) {             /* L y = -b' */
        double t = -bp[i];
        for (int k = 0; k < i; ++k) t -= L[IDX(i, k, n)] * y[k];
        y[i] = t / L[IDX(i, i, n)];
    }
    for (int i = n - 1; i >= 0; --i) {        /* L^T x = y */
        double t = y[i];
        for (int k = i + 1; k < n; ++k) t -= L[IDX(k, i, n)] * x0[k];
        x0[i] = t / L[IDX(i, i, n)];
    }
    free(L);
    free(y);
    return 0;
}

/* Problem (p): h(x,p) = x^T Q x + b^T x + sum p_i (x_i - x_i^2); its gradient
 * g = 2 (Q - P*) x + (b + p) as used in Eq. (dp1) and Alg. 2 (g^k). */
double orc_penalized(int n, const double* Q, const double* b, const double* p, const double* x,
                     double* g)
{
    double h = 0.0;
    for (int i = 0; i < n; ++i) {
        double qx = 0.0;
        for (int j = 0; j < n; ++j) qx += Q[IDX(i, j, n)] * x[j];
        double bi = b ? b[i] : 0.0;
        double pi = p ? p[i] : 0.0;
        h += x[i] * qx + bi * x[i] + pi * (x[i] - x[i] * x[i]);
        if (g) g[i] = 2.0 * qx - 2.0 * pi * x[i] + bi + pi;
    }
    return h;
}

/* Sec. 3.3, Eq. (cret): on I = {0<x<1} the gradient must vanish, on J = {x=0} it
 * must be >= 0 and on K = {x=1} it must be <= 0; cret is the largest violation. */
double orc_kkt_residual(int n, const double* x, const double* g)
{
    double c = 0.0;
    for (int i = 0; i < n; ++i) {
        double v;
        if (x[i] > 0.0 && x[i] < 1.0) v = fabs(g[i]);
        else if (x[i] <= 0.0) v = g[i] < 0.0 ? -g[i] : 0.0;
        else v = g[i] > 0.0 ? g[i] : 0.0;
        if (v > c) c = v;
    }
    return c;
}

/* Sec. 3.3: rho = max{1, |2(Q - P*)|, |b + p|} with |.| the largest absolute entry. */
double orc_rho(int n, const double* Q, const double* b, const double* p)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double q = Q[IDX(i, j, n)] - (i == j && p ? p[i] : 0.0);
            if (fabs(2.0 * q) > r) r = fabs(2.0 * q);
        }
        double bb = (b ? b[i] : 0.0) + (p ? p[i] : 0.0);
        if (fabs(bb) > r) r = fabs(bb);
    }
    return r;
}

/* Number of eigenvalues of the tridiagonal (a, e) strictly below x (Sturm count). */
static int sturm_count(int m, const double* a, const double* e, double x)
{
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0.0) ++cnt;
    for (int i = 1; i < m; ++i) {
        if (q == 0.0) q = DBL_EPSILON * (fabs(e[i - 1]) + DBL_MIN);
        q = (a[i] - x) - e[i - 1] * e[i - 1] / q;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

/* lambda_min of Eq. (eq:alpha): Householder reduction to tridiagonal form, then
 * bisection on the Sturm count (textbook dense symmetric eigenvalue method). */
double orc_lambda_min(int m, double* A)
{
    if (m <= 0) return 0.0;
    if (m == 1) return A[0];
    double* v = (double*)malloc((size_t)m * sizeof(double));
    double* w = (double*)malloc((size_t)m * sizeof(double));
    double* a = (double*)malloc((size_t)m * sizeof(double));
    double* e = (double*)calloc((size_t)m, sizeof(double));
    for (int k = 0; k + 2 < m; ++k) {
        int len = m - k - 1;                  /* column k below the diagonal */
        double nrm2 = 0.0;
        for (int i = 0; i < len; ++i) {
            v[i] = A[IDX(k + 1 + i, k, m)];
            nrm2 += v[i] * v[i];
        }
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) { e[k] = 0.0; continue; }
        double sgn = v[0] >= 0.0 ? 1.0 : -1.0;
        v[0] += sgn * nrm;
        double vv = 0.0;
        for (int i = 0; i < len; ++i) vv += v[i] * v[i];
        double beta = 2.0 / vv;
        /* w = beta S v - (beta/2)(v^T beta S v) v, S the trailing block */
        double pv = 0.0;
        for (int i = 0; i < len; ++i) {
            double s = 0.0;
            for (int j = 0; j < len; ++j) s += A[IDX(k + 1 + i, k + 1 + j, m)] * v[j];
            w[i] = beta * s;
            pv += w[i] * v[i];
        }
        double K = 0.5 * beta * pv;
        for (int i = 0; i < len; ++i) w[i] -= K * v[i];
        for (int i = 0; i < len; ++i)
            for (int j = 0; j < len; ++j)
                A[IDX(k + 1 + i, k + 1 + j, m)] -= v[i] * w[j] + w[i] * v[j];
        e[k] = -sgn * nrm;
    }
    e[m - 2] = A[IDX(m - 1, m - 2, m)];
    for (int i = 0; i < m; ++i) a[i] = A[IDX(i, i, m)];
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
        if (a[i] - r < lo) lo = a[i] - r;
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 300; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(m, a, e, mid) >= 1) hi = mid; else lo = mid;
    }
    free(v); free(w); free(a); free(e);
    return 0.5 * (lo + hi);
}

/* Sec. 3.4, Lemma 3.1 and Eq. (eq:alpha1): alpha = eta * lambda_min of the matrix
 * Z^-1/2 Qbar_II Z^-1/2 with z = x - x^2 and I the interior coordinates. */
double orc_penalty_step(int n, const double* Qp, const double* bp, const double* p, const double* x,
                        const orc_opts* o, int consecutive, int* n_active, double* lambda, int* fallback)
{
    int* idx = (int*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    double* rz = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int m = 0;
    for (int i = 0; i < n; ++i) {
        double z = x[i] - x[i] * x[i];
        if (z > o->tau_z) { idx[m] = i; rz[m] = 1.0 / sqrt(z); ++m; }
    }
    *n_active = m;
    *fallback = 0;
    if (m == 0) { free(idx); free(rz); *lambda = 0.0; return 0.0; }
    double* A = (double*)malloc((size_t)m * m * sizeof(double));
    double qmax = 1.0;
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) {
            int i = idx[a], j = idx[c];
            double q = Qp[IDX(i, j, n)] - (i == j ? p[i] : 0.0);
            if (fabs(q) > qmax) qmax = fabs(q);
            A[IDX(a, c, m)] = rz[a] * q * rz[c];
        }
    double lam = orc_lambda_min(m, A);
    *lambda = lam;
    /* Floor: the smallest curvature change the stopping test of Eq. (cret) can
     * resolve, lambda_floor_rel * delta * rho in the Z-scaled units of Eq. (eq:alpha).
     * Below it (flat or negative curvature on I) the floor is used instead, doubled
     * for every consecutive outer step that needed it. */
    double floor = o->lambda_floor_rel * o->tol_inner * orc_rho(n, Qp, bp, p);
    double alpha;
    if (lam > floor) alpha = o->eta * lam;
    else { alpha = o->eta * ldexp(floor, consecutive < 60 ? consecutive : 60); *fallback = 1; }
    (void)qmax;
    free(A); free(idx); free(rz);
    return alpha;
}

static void penalized_gradient(int n, const double* Qp, const double* bp, const double* p,
                               const double* x, double* g)
{
    for (int i = 0; i < n; ++i) {
        double qx = 0.0;
        for (int j = 0; j < n; ++j) qx += Qp[IDX(i, j, n)] * x[j];
        g[i] = 2.0 * qx - 2.0 * p[i] * x[i] + bp[i] + p[i];
    }
}

static double clip01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Rounding model of orc_opts.fp32_noise: SplitMix64 (Steele, Lea, Flood 2014) of a key, mapped
 * to a uniform number in [-1, 1]. */
static double noise_uniform(unsigned long long seed, long long count, int i)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(count * 1000003LL + i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static void noise_gradient(int n, const double* Qp, const double* bp, const double* p, const double* x,
                           double* g, const orc_opts* o, long long count)
{
    if (!(o->fp32_noise > 0.0)) return;
    for (int i = 0; i < n; ++i) {
        /* the terms of g_i = 2 sum_{j != i} Q'_ij x_j + (d_i - p_i)(2 x_i - 1) + (d_i + b'_i),
         * where the gamma-sized parts of 2 (d_i - p_i) x_i and b'_i + p_i cancel exactly */
        double s = 0.0;
        for (int j = 0; j < n; ++j)
            if (j != i) s += fabs(Qp[IDX(i, j, n)] * x[j]);
        const double d = Qp[IDX(i, i, n)];
        s = 2.0 * s + fabs((d - p[i]) * (2.0 * x[i] - 1.0)) + fabs(d + bp[i]);
        g[i] += o->fp32_noise * noise_uniform(o->noise_seed, count, i) * s;
    }
}

static void noise_iterate(int n, double* x, const orc_opts* o, long long count)
{
    if (!(o->fp32_noise > 0.0)) return;
    for (int i = 0; i < n; ++i)
        x[i] = clip01(x[i] * (1.0 + o->fp32_noise * noise_uniform(o->noise_seed ^ 0x5DEECE66Dull, count, i)));
}

/* Alg. 2 (PABB): x^{k+1} = P(x^k - alpha_k g^k), Eq. (x2), with the alternating
 * Barzilai-Borwein step of Eq. (bb1); Alg. 1 (PPA): x^{k+1} = P(x^k - g^k/(2 h_p)),
 * Eq. (x1), with H_p of Sec. 3.1.  Both stop on Eq. (cret). */
int orc_inner(int n, const double* Qp, const double* bp, const double* p, double* x,
              const orc_opts* o, int trace_len, double* trace_x, double* trace_alpha,
              long long* grad_evals, int* exit_code)
{
    double* g = (double*)malloc((size_t)n * sizeof(double));
    double* xp = (double*)malloc((size_t)n * sizeof(double));
    double* gp = (double*)malloc((size_t)n * sizeof(double));
    double* hp = (double*)malloc((size_t)n * sizeof(double));
    penalized_gradient(n, Qp, bp, p, x, g);
    noise_gradient(n, Qp, bp, p, x, g, o, 0);
    long long ge = 1;
    double rho = orc_rho(n, Qp, bp, p);
    double alpha = 0.0;
    if (o->method == 0) {                      /* alpha_0 = 1 / (2 ||Qbar||_inf) */
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) {
            double r = 0.0;
            for (int j = 0; j < n; ++j) r += fabs(Qp[IDX(i, j, n)] - (i == j ? p[i] : 0.0));
            if (r > nrm) nrm = r;
        }
        alpha = nrm > 0.0 ? 1.0 / (2.0 * nrm) : 1.0;
    } else {                                   /* h_p = max(sum_i |Q_ji| - p_j, eps) */
        double rmax = 1.0;
        for (int i = 0; i < n; ++i) {
            double r = 0.0;
            for (int j = 0; j < n; ++j) r += fabs(Qp[IDX(i, j, n)]);
            hp[i] = r;
            if (r > rmax) rmax = r;
        }
        double eps = o->eps_hp_rel * rmax;
        for (int i = 0; i < n; ++i) hp[i] = fmax(hp[i] - p[i], eps);
    }
    int k = 0, code = 1;
    for (;;) {
        if (trace_x && k < trace_len) memcpy(trace_x + (size_t)k * n, x, (size_t)n * sizeof(double));
        if (orc_kkt_residual(n, x, g) / rho < o->tol_inner) { code = 0; break; }
        if (k >= o->max_inner) { code = 1; break; }
        int moved = 0;
        if (o->method == 0) {
            if (k >= 1) {
                double ss = 0.0, sy = 0.0, yy = 0.0;
                for (int i = 0; i < n; ++i) {
                    double s = x[i] - xp[i], y = g[i] - gp[i];
                    ss += s * s; sy += s * y; yy += y * y;
                }
                if (ss == 0.0) { code = 2; break; }
                double a = (k % 2 == 1) ? ss / sy : sy / yy;
                if (!(sy > 0.0) || !isfinite(a)) a = alpha;
                if (a < o->alpha_min) a = o->alpha_min;
                if (a > o->alpha_max) a = o->alpha_max;
                alpha = a;
            }
            if (trace_alpha && k < trace_len) trace_alpha[k] = alpha;
            for (int i = 0; i < n; ++i) {
                xp[i] = x[i];
                gp[i] = g[i];
                x[i] = clip01(x[i] - alpha * g[i]);
                moved |= (x[i] != xp[i]);
            }
        } else {
            if (trace_alpha && k < trace_len) trace_alpha[k] = NAN;
            for (int i = 0; i < n; ++i) {
                double xn = clip01(x[i] - g[i] / (2.0 * hp[i]));
                moved |= (xn != x[i]);
                x[i] = xn;
            }
        }
        ++k;
        if (!moved) { code = 2; break; }
        noise_iterate(n, x, o, ge);
        penalized_gradient(n, Qp, bp, p, x, g);
        noise_gradient(n, Qp, bp, p, x, g, o, ge);
        ++ge;
    }
    free(g); free(xp); free(gp); free(hp);
    if (grad_evals) *grad_evals = ge;
    if (exit_code) *exit_code = code;
    return k;
}

static double binarity(int n, const double* x)
{
    double m = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = fmin(x[i], 1.0 - x[i]);
        if (d > m) m = d;
    }
    return m;
}

/* Alg. 3: initialization (Sec. 3.5), then penalty update (Eq. (pp1), (eq:alpha1))
 * followed by a subproblem solve, until x is binary; the best rounded point is kept
 * (Sec. 3.4: "the best value of x"). */
int orc_solve(int n, const double* Q, const double* b, const double* mu, const double* x_start,
              const orc_opts* o, uint8_t* x_best, double* f_best, orc_stats* st, int* inner_hist,
              double* p_out)
{
    memset(st, 0, sizeof(*st));
    if (n <= 0) { st->status = -1; return -1; }
    double* Qp = (double*)malloc((size_t)n * n * sizeof(double));
    double* bp = (double*)malloc((size_t)n * sizeof(double));
    double* gam = (double*)malloc((size_t)n * sizeof(double));
    double* x = (double*)malloc((size_t)n * sizeof(double));
    double* p = (double*)calloc((size_t)n, sizeof(double));
    uint8_t* xr = (uint8_t*)malloc((size_t)n);
    orc_reformulate(n, Q, b, mu, o->gamma_margin, Qp, bp, gam);
    if (x_start) {
        memcpy(x, x_start, (size_t)n * sizeof(double));
    } else if (orc_initial_point(n, Qp, bp, x) != 0) {
        st->status = -2;
        free(Qp); free(bp); free(gam); free(x); free(p); free(xr);
        return -2;
    }
    double best = INFINITY;
    int s = 0, consec = 0;
    for (;;) {
        for (int i = 0; i < n; ++i) xr[i] = x[i] > 0.5;
        double f = orc_objective(n, Q, b, xr);
        if (f < best) {
            best = f;
            memcpy(x_best, xr, (size_t)n);
            st->best_outer = s;
        }
        if (binarity(n, x) <= o->tol_outer) { st->status = 0; break; }
        if (s >= o->max_outer) { st->status = 1; break; }
        int m = 0, fb = 0;
        double lam = 0.0;
        double alpha = orc_penalty_step(n, Qp, bp, p, x, o, consec, &m, &lam, &fb);
        if (m == 0) { st->status = 0; break; }
        st->n_fallback += fb;
        consec = fb ? consec + 1 : 0;
        for (int i = 0; i < n; ++i) p[i] += alpha * (x[i] - x[i] * x[i]);
        long long ge = 0;
        int code = 0;
        int k = orc_inner(n, Qp, bp, p, x, o, 0, NULL, NULL, &ge, &code);
        if (inner_hist) inner_hist[s] = k;
        st->inner_total += k;
        st->grad_evals += ge;
        ++s;
    }
    st->outer = s;
    st->final_binarity = binarity(n, x);
    *f_best = best;
    if (p_out) memcpy(p_out, p, (size_t)n * sizeof(double));
    free(Qp); free(bp); free(gam); free(x); free(p); free(xr);
    return st->status;
}
