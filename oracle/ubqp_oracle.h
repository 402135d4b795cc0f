/*
 * FP64 CPU oracle of the vectorized PSDP method for UBQP (arXiv 2408.04875).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 * The product path never links, loads or calls it, and it shares no code with it.
 *
 * Plain loops in double precision, no BLAS, no blocking or reordering beyond what
 * the paper's definitions state.  Equation labels are the paper's LaTeX labels.
 *
 * Readings of points the paper leaves open are fixed in orc_opts_default():
 *   - the subproblem of outer step s is solved with the updated penalty p^{s+1};
 *   - the outer test uses the distance to the nearest binary point;
 *   - the KKT residual uses the true gradient 2*Qbar*x + bbar on I, J and K;
 *   - rho uses the largest absolute entry of 2*Qbar and of bbar;
 *   - eta = 0.9, gamma_i = 2*sum_j |Q_ij| + |b_i| + 1 (perturbed Q);
 *   - BB: alpha_0 = 1 / (2 ||Qbar||_inf), k odd -> BB1, k even -> BB2,
 *     s^T y <= 0 or non-finite -> previous step, clamp to [alpha_min, alpha_max],
 *     s = 0 -> stop;
 *   - lambda_min taken over I_alpha = {i : x_i - x_i^2 > tau_z};
 *   - lambda_min below the resolution F = 4 * delta * rho of the stopping test
 *     (flat or negative curvature on I) -> alpha = eta * F * 2^c, c the number of
 *     consecutive outer steps that took this branch;
 *   - every rounded iterate x^s (s = 0, 1, ...) is a candidate for the best value.
 */
#ifndef UBQP_ORACLE_H
#define UBQP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int method;             /* 0 = PABB (Alg. 2), 1 = PPA (Alg. 1)                   */
    int max_outer;          /* penalty updates, Sec. 5: 1000                          */
    int max_inner;          /* subproblem iterations, Sec. 5: 10000                   */
    double tol_inner;       /* delta in Eq. (cret): 1e-5                              */
    double tol_outer;       /* Alg. 3 while-test threshold: 1e-5                      */
    double eta;             /* Eq. (eq:alpha1), 0 < eta < 1                           */
    double gamma_margin;    /* Eq. (gamma) strict inequality margin                   */
    double alpha_min;       /* BB step clamp                                          */
    double alpha_max;
    double tau_z;           /* z_i > tau_z defines the index set of Eq. (eq:alpha)    */
    double eps_hp_rel;      /* PPA epsilon = eps_hp_rel * max(1, max_j r_j), Sec. 3.1 */
    double lambda_floor_rel;/* floor F = lambda_floor_rel * tol_inner * rho (Sec. 3.4)  */
    /* Rounding model for sensitivity studies (tests only; 0 = off, the default, and then
     * nothing below changes the arithmetic): after every gradient evaluation of orc_inner,
     * g_i += fp32_noise * r * s_i with s_i = 2 sum_{j != i} |Q'_ij x_j| + |(d_i - p_i)(2 x_i - 1)|
     * + |d_i + b'_i| (d = diag Q'; the terms of g_i once the gamma-sized parts of
     * 2 (d_i - p_i) x_i and b'_i + p_i cancel), and after every projected step
     * x_i <- clip(x_i (1 + fp32_noise * r')); r, r' uniform in [-1, 1] from SplitMix64 keyed
     * by (noise_seed, evaluation, i). */
    double fp32_noise;
    unsigned long long noise_seed;
} orc_opts;

typedef struct {
    int outer;              /* subproblems solved                                     */
    long long inner_total;  /* projected steps over all subproblems                   */
    long long grad_evals;   /* gradient evaluations over all subproblems              */
    int best_outer;         /* outer step whose rounded point gave the best value     */
    int n_fallback;         /* penalty steps that used the fallback alpha             */
    int status;             /* 0 ok, 1 outer cap reached, <0 error                    */
    double final_binarity;  /* max_i min(x_i, 1 - x_i) at exit                         */
} orc_stats;

void orc_opts_default(orc_opts* o);

/* f(x) = x^T Q x + b^T x for x in {0,1}^n (Eq. (bqp)); b may be NULL. */
double orc_objective(int n, const double* Q, const double* b, const uint8_t* x);

/* Sec. 3.5: Q' = Q + mu + Diag(gamma), b' = b - gamma with
 * gamma_i = 2 sum_j |(Q+mu)_ij| + |b_i| + margin.  mu and b may be NULL. */
void orc_reformulate(int n, const double* Q, const double* b, const double* mu, double margin,
                     double* Qp, double* bp, double* gamma);

/* Eq. (gamma): solve 2 Q' x = -b' by Cholesky.  Returns 0, or -1 if Q' is not SPD. */
int orc_initial_point(int n, const double* Qp, const double* bp, double* x0);

/* h(x,p) = x^T Q x + b^T x + sum_i p_i (x_i - x_i^2) (Sec. 4.1, problem (p)) and
 * its gradient g = 2 (Q - Diag p) x + (b + p) (Sec. 3.1).  g may be NULL. */
double orc_penalized(int n, const double* Q, const double* b, const double* p, const double* x,
                     double* g);

/* Eq. (cret): the KKT residual cret for gradient g at x. */
double orc_kkt_residual(int n, const double* x, const double* g);

/* rho = max{1, max|2 Qbar_ij|, max|bbar_i|}, Qbar = Q - Diag p, bbar = b + p. */
double orc_rho(int n, const double* Q, const double* b, const double* p);

/* Smallest eigenvalue of the dense symmetric m x m matrix A (row-major, destroyed):
 * Householder tridiagonalization followed by Sturm-sequence bisection. */
double orc_lambda_min(int m, double* A);

/* Sec. 3.4: alpha = eta * lambda_min(Z^-1/2 Qbar_II Z^-1/2) over I_alpha, or, when
 * lambda_min <= F = lambda_floor_rel * tol_inner * rho, alpha = eta * F * 2^consecutive
 * (consecutive = floor steps taken in a row before this one).
 * Returns the step; *n_active receives |I_alpha|, *lambda the eigenvalue,
 * *fallback is set to 1 when the floor rule was used. */
double orc_penalty_step(int n, const double* Qp, const double* bp, const double* p, const double* x,
                        const orc_opts* o, int consecutive, int* n_active, double* lambda,
                        int* fallback);

/* Alg. 2 (PABB) or Alg. 1 (PPA) on problem (p1) with fixed p, starting from x (updated
 * in place).  Traces: iterate k is written to trace_x[k*n..] for k < trace_len, and
 * the step used at iteration k to trace_alpha[k] (either may be NULL).
 * Returns the number of projected steps taken; *grad_evals the gradient evaluations;
 * *exit_code: 0 KKT test met, 1 iteration cap, 2 zero step. */
int orc_inner(int n, const double* Qp, const double* bp, const double* p, double* x,
              const orc_opts* o, int trace_len, double* trace_x, double* trace_alpha,
              long long* grad_evals, int* exit_code);

/* Alg. 3: the whole method.  Q, b are the original data (b may be NULL); mu is the
 * symmetric perturbation (may be NULL).  x_start (may be NULL) replaces the x^0 of
 * Eq. (gamma) as the first iterate.  Writes the best rounded point and its exact
 * objective.  inner_hist (may be NULL, length >= max_outer) receives the inner step
 * count of every subproblem; p_out (may be NULL, length n) the penalty vector p of the
 * last subproblem. */
int orc_solve(int n, const double* Q, const double* b, const double* mu, const double* x_start,
              const orc_opts* o, uint8_t* x_best, double* f_best, orc_stats* st, int* inner_hist,
              double* p_out);

#ifdef __cplusplus
}
#endif
#endif
