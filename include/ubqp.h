/*
 * ubqp.h - C ABI of the GB300 (sm_103a) implementation of the vectorized
 * positive-semidefinite-penalty (PSDP) method for unconstrained binary quadratic
 * programs, arXiv 2408.04875 (Huo & Gu):
 *
 *     min  f(x) = x^T Q x + b^T x     over x in {0,1}^n,  Q symmetric   (Eq. (bqp))
 *
 * The library runs Alg. 3 of the paper on one GPU: initialization (Sec. 3.5:
 * reformulation with gamma, random symmetric perturbation, x^0 from Eq. (gamma)),
 * the penalty update p += alpha z with alpha from Lemma 3.1 / Eq. (eq:alpha1), the
 * subproblem solver (Alg. 2, projected alternating Barzilai-Borwein, or Alg. 1,
 * proximal point) with the KKT stopping test of Eq. (cret), then rounding and exact
 * evaluation of every candidate, keeping the best.
 *
 * Conventions shared by all entry points
 *   - Matrices are dense, row-major, n x n, FP64 unless stated otherwise.
 *   - Pointers may be host or device memory unless stated otherwise; the library
 *     detects which with cudaPointerGetAttributes.  It never keeps a caller pointer
 *     after returning and never frees caller memory.
 *   - Every call returns a ubqp_status.  Negative values are errors (outputs are
 *     then unspecified); positive values are warnings (outputs valid).  Detail for the
 *     last failing call of the calling thread is available from ubqp_last_error().
 *     The library never aborts, traps or prints.
 *   - All GPU work runs on opts->stream (NULL = the legacy default stream) of the
 *     current device; the entry points synchronize that stream before returning.
 *   - Every device-side wait is bounded; a wait that runs out returns UBQP_ETIMEOUT
 *     and leaves the device usable.
 */
#ifndef UBQP_H
#define UBQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UBQP_OK = 0,
    UBQP_EINVAL = -1,      /* bad argument (size, NULL pointer, option out of range) */
    UBQP_ENOTSYM = -2,     /* Q is not symmetric                                     */
    UBQP_ENONFINITE = -3,  /* Q or b holds NaN or Inf                                */
    UBQP_ECUDA = -4,       /* a CUDA runtime or driver call failed                   */
    UBQP_ENOMEM = -5,      /* device allocation failed                               */
    UBQP_ETIMEOUT = -6,    /* a bounded device wait ran out                          */
    UBQP_ENOTSUP = -7,     /* request not supported on this device / configuration  */
    UBQP_EMAXITER = 1      /* warning: some instance hit max_outer; results valid    */
} ubqp_status;

enum { UBQP_PABB = 0, UBQP_PPA = 1 };                 /* subproblem solver        */
enum { UBQP_FP32 = 0, UBQP_BF16X2_TC = 1, UBQP_BF16_TC = 2 };  /* matvec precision */
enum { UBQP_DTYPE_F32 = 0, UBQP_DTYPE_F64 = 1 };

#define UBQP_HIST_BINS 101   /* inner-iteration histogram: bins of 100 steps, last = 10000+ */

/* Counters of one solve (sums over every lane = instance x start). */
typedef struct {
    int64_t inner_iters;     /* gradient evaluations of the subproblem solver         */
    int64_t inner_steps;     /* projected steps (Alg. 1/2 iterations)                 */
    int64_t var_updates;     /* sum over lanes of inner_iters * n                     */
    int64_t outer_steps;     /* subproblems solved (penalty updates)                  */
    int64_t lobpcg_iters;    /* eigen-solver iterations for lambda_min                */
    int64_t jacobi_iters;    /* sweeps spent on x^0                                   */
    int64_t floor_steps;     /* penalty steps that used the resolution floor          */
    int64_t ticks;           /* device ticks (one matvec pass over all active lanes)  */
    int64_t lanes;           /* instance x start pairs                                */
    int64_t lanes_capped;    /* lanes that stopped at max_outer                        */
    double ms_device;        /* device time of the iteration loop (CUDA events)        */
    double ms_total;         /* whole call, host wall clock                           */
    double phase_a_ms;       /* summed duration of the matvec (phase A) launches,      */
                             /* CUDA events around each launch (profile_kernels only)  */
    int64_t phase_a_launches;/* phase-A launches timed                                 */
    int64_t phase_a_bytes;   /* algorithmic bytes of those launches: stored matrix     */
                             /* entries of every active lane once, plus its vectors    */
    int64_t kernel_launches; /* launches of this library's kernels during the call      */
    double ms_to_target;     /* device time until some lane's best objective reached    */
                             /* opts->target_objective (-1: not reached / not set)      */
    int64_t phase_a_flops;   /* algorithmic flops of the tensor-core launches timed     */
    int32_t cluster_size;    /* CTAs per cluster of the tensor-core launches (0: none)  */
    int32_t gemv_kernel;     /* scheduler that ran the FP32 lanes: 1 lock-step, 2 lane  */
                             /* loop, 3 single-lane kernel (0: tensor-core lanes)       */
    int32_t restarts;        /* starts per instance that ran (the tuner's pick when     */
                             /* opts->restarts == 0)                                    */
    float restart_probe_us[5]; /* restart tuner: step time measured with 1, 8, 32, 64  */
                             /* and 128 starts per instance (0 when not tuned)          */
    int32_t tc_kernel;       /* tensor-core contraction that ran: 1 split-K clusters,   */
                             /* 2 persistent (many tiles), 0 none                       */
    int32_t sym_storage;     /* 1 when the FP32 lanes ran on the symmetric tiles        */
    int64_t inner_hist[UBQP_HIST_BINS]; /* projected steps per subproblem (Fig. 5)   */
    int64_t alg_bytes;       /* sparse-minimum bytes of every matrix-vector product run:  */
                             /* sum over lanes of steps x (6 nnz(Q_off) + 32 n), i.e. the */
                             /* stored off-diagonal entries as 4-byte values with 2-byte  */
                             /* column indices plus 8 vectors of n floats per step        */
    int64_t alg_flops;       /* sum over lanes of steps x 2 nnz(Q_off)                    */
    float cluster_probe_us[9]; /* tensor-core form tuner (tc_cluster = 0): contraction time */
                             /* of the persistent many-tile kernel [0] and of split-K over */
                             /* S = 1..8 CTAs [S], best of three launches (0: not probed)  */
    int32_t cluster_tuned;   /* 0: rule or caller's tc_cluster, 1: measured in this call,  */
                             /* 2: taken from the cache (see tc_cluster)                  */
    int32_t storage;         /* Q'_off as read by phase A: 0 dense FP32 rows, 1 symmetric  */
                             /* tiles, 2 sliced rows (sparse), 3 BF16 tensor-core tiles    */
} ubqp_stats;

/* Options; ubqp_opts_default() fills the paper's settings and this library's readings
 * of the points the paper leaves open. */
typedef struct {
    int method;              /* UBQP_PABB (Alg. 2, default) or UBQP_PPA (Alg. 1)     */
    int max_outer;           /* 1000 penalty updates (Sec. 5)                          */
    int max_inner;           /* 10000 subproblem iterations (Sec. 5)                   */
    double tol_inner;        /* delta of Eq. (cret): 1e-5                              */
    double tol_outer;        /* Alg. 3 while-test on max_i min(x_i, 1-x_i): 1e-5       */
    double eta;              /* Eq. (eq:alpha1), 0 < eta < 1: 0.9                      */
    double gamma_margin;     /* gamma_i = 2 sum_j |Q_ij| + |b_i| + margin: 1.0         */
    double alpha_min;        /* clamp of the BB step: 1e-10                             */
    double alpha_max;        /*                        1e10                             */
    double tau_z;            /* coordinates with x - x^2 > tau_z enter lambda_min: 1e-12 */
    double eps_hp_rel;       /* PPA epsilon relative to max row sum: 1e-8              */
    double lambda_floor_rel; /* resolution floor F = this * tol_inner * rho: 4.0        */
    double sigma_rel;        /* perturbation std-dev / max|Q_ij| (i != j): 1e-3; 0 = off */
    uint64_t seed;           /* seeds the library's own draws (perturbation, starts)  */
    int restarts;            /* starts per instance: 1 = x^0 of Eq. (gamma) only;      */
                             /* R > 1 adds R-1 starts uniform in [0,1]^n; 0 = chosen  */
                             /* by the restart tuner from {1, 8, 32, 64, 128}: each    */
                             /* count runs a 32-step probe on the real batch and the   */
                             /* largest whose step time is at most twice that of one  */
                             /* start wins (needs x_starts == NULL)                    */
    int precision;           /* UBQP_FP32 (default), UBQP_BF16X2_TC, UBQP_BF16_TC      */
    int lobpcg_max_iter;     /* cap of the lambda_min eigen-solver: 256                */
    double lobpcg_tol;       /* relative change of the Ritz value to stop: 1e-7 (the   */
                             /* Ritz value is an upper bound of lambda_min, so a loose */
                             /* stop overstates alpha); tensor-core lanes stop at      */
                             /* max(lobpcg_tol, 1e-5), their products' resolution      */
    int jacobi_max_iter;     /* sweeps for x^0: 60                                      */
    int max_ticks_per_sync;  /* ticks launched between host checks: 64                 */
    int profile_kernels;     /* 1: time every phase-A launch with CUDA events; 2: also  */
                             /* keep a per-tick timeline (ubqp_profile_timeline): 0     */
    int stop_at_target;      /* 1: stop once target_objective is reached: 0            */
    int tc_cluster;          /* CTAs splitting K in the tensor-core kernel, 1..8;      */
                             /* 0 = chosen by measurement: the contraction alone is     */
                             /* timed with every feasible S and with the persistent      */
                             /* many-tile kernel, on the call's operands, and the        */
                             /* fastest kept; the choice is cached per shape in the      */
                             /* process and, when the environment variable               */
                             /* UBQP_TUNE_CACHE names a file, in that JSON file          */
    int gemv_kernel;         /* scheduler of the FP32 lanes: 1 lock-step (one launch   */
                             /* per step of all lanes), 2 persistent lane loop (lanes  */
                             /* advance independently inside one launch), 3 single-lane */
                             /* persistent kernel (many steps per cooperative launch;  */
                             /* each lane on its own group of CTAs with a bounded group */
                             /* barrier, one per PABB step; with more lanes than       */
                             /* resident CTAs, one-CTA groups run several lanes in      */
                             /* turn); 0 = 3 for one lane and for lanes on the sliced   */
                             /* storage whose groups fit with at most 5 slices per CTA, */
                             /* else 2 for 4 or more lanes, else 1 (1 when              */
                             /* profile_kernels == 2); UBQP_ENOTSUP when 3 is asked for */
                             /* and a lane's two vectors exceed 200 KiB of shared memory */
    int lane_budget;         /* lane loop and single-lane kernel: steps per lane (per   */
                             /* group) between host checks; 0 = 1024                    */
    int rows_per_item;       /* FP32 lanes: matrix rows per work item, 8..256 (a multiple */
                             /* of 8); 0 = chosen from the batch size                  */
    int sym_storage;         /* FP32 lanes on the lane loop: 1 = store only the upper   */
                             /* triangle of Q'_off (128 x 128 tiles; each step reads    */
                             /* about half the bytes), 0 = dense rows: 1                */
    int wait_limit_us;       /* lane loop and single-lane kernel: limit of one wait of a  */
                             /* CTA (for its next ring slot / at a grid barrier), in     */
                             /* microseconds; a wait that runs out ends the call with    */
                             /* UBQP_ETIMEOUT and leaves the device usable; 0 = 5 s      */
    int tc_fuse;             /* tensor-core lanes: 1 = the contraction's epilogue warps run */
                             /* each lane's update as soon as its last M tile is done (one */
                             /* launch per step; lanes of at most 32 M tiles), 0 = a      */
                             /* separate update launch (one CTA per lane) after every     */
                             /* contraction: 0 (the lanes of an N tile all finish on one  */
                             /* tile, so fused updates serialize in one CTA)              */
    int sparse_storage;      /* FP32 lanes: Q'_off in sliced row storage (32-row slices of */
                             /* the stored entries: 4-byte value, 2-byte column), read by  */
                             /* every scheduler; 0 = when its bytes are fewer than the     */
                             /* symmetric tiles' (stored off-diagonal entries < n^2 / 3),  */
                             /* 1 = always, 2 = never: 0                                  */
    double target_objective; /* objective to time against (used when finite)           */
    void* stream;            /* cudaStream_t, NULL = default stream                    */
    const double* const* mu; /* optional perturbations, one n x n matrix per instance   */
                             /* (symmetric); NULL = drawn from seed when sigma_rel > 0 */
    const double* const* x_starts; /* optional extra starts, one (R-1) x n block per   */
                             /* instance; NULL = drawn from seed                        */
    ubqp_stats* stats;       /* optional output (host memory)                          */
} ubqp_opts;

/* Fills *o with the defaults listed above. */
void ubqp_opts_default(ubqp_opts* o);

/* Human-readable name of a status code (static storage). */
const char* ubqp_status_string(int status);

/* Detail on the last error of the calling thread (static thread-local storage). */
const char* ubqp_last_error(void);

/*
 * ubqp_solve - Alg. 3 for one instance.
 *   Q      n x n symmetric (checked: |Q_ij - Q_ji| <= 1e-12 max|Q|), host or device.
 *   b      n, host or device; NULL means b = 0.
 *   n      1 <= n <= 65536.
 *   o      options; NULL means defaults.
 *   x_out  n bytes (0/1), host or device: the best rounded point found.
 *   obj_out 1 double, host or device: f(x_out) of the ORIGINAL Q, b, evaluated in FP64
 *          (exact for integer data with |f| < 2^53).
 * Returns UBQP_OK, UBQP_EMAXITER (warning), or a negative error.
 * The same as ubqp_solve_batched with num = 1.
 */
int ubqp_solve(const double* Q, const double* b, int64_t n, const ubqp_opts* o,
               uint8_t* x_out, double* obj_out);

/*
 * ubqp_solve_batched - Alg. 3 for num independent instances of uneven size, each with
 * o->restarts starts, all advanced together on the device (one lane per instance x
 * start; lanes of one instance share its Q).
 *   num    >= 1 instances;  n[i], Q[i], b[i] (b may be NULL or hold NULL entries) as
 *          in ubqp_solve.
 *   x_out[i] n[i] bytes, obj_out num doubles: per instance, the best rounded point over
 *          all of its starts and outer steps and its exact objective.
 * With o->precision = UBQP_BF16X2_TC / UBQP_BF16_TC the matvecs of all starts of an
 * instance run as one BF16 tensor-core contraction (Q off-diagonal in BF16, the iterate
 * split into two BF16 terms for X2, FP32 accumulation); the perturbation then touches
 * only the diagonal (kept in FP32), since BF16 cannot carry it off the diagonal.  These
 * precisions require every off-diagonal entry to be exactly representable in BF16 (for
 * example integers of magnitude <= 256), so that rounded points are evaluated exactly;
 * otherwise the call returns UBQP_ENOTSUP.
 */
int ubqp_solve_batched(int32_t num, const int64_t* n, const double* const* Q,
                       const double* const* b, const ubqp_opts* o, uint8_t* const* x_out,
                       double* obj_out);

/*
 * ubqp_penalized_eval - the penalized objective of Sec. 4.1, problem (p), and its
 * gradient (Sec. 3.1, used as g^k in Alg. 2), for `batch` points sharing Q, b, p:
 *     h_r = x_r^T Q x_r + b^T x_r + sum_i p_i (x_ri - x_ri^2)
 *     g_r = 2 (Q - Diag p) x_r + b + p
 * All pointers are DEVICE memory of element type dtype (UBQP_DTYPE_F32 / _F64), each
 * aligned to its element size:
 *   Q n x n row-major (no padding), b and p n (either may be NULL = 0), x batch x n
 *   row-major, h_out batch (may be NULL), g_out batch x n (may be NULL).
 * 1 <= n <= 65536 and one point must fit in shared memory (n * element size <= 227 KiB,
 * else UBQP_ENOTSUP).  stream: cudaStream_t (NULL = default).
 * Runs the kernel of the inner loop's matrix-vector products (the lock-step GEMV kernel:
 * the same row dot with compensated FP32 sums, here on the caller's rows) with the
 * gradient epilogue; the FP64 dtype runs the same kernel source on FP64 data.  h is summed
 * in FP64.  Scratch (descriptors, work items, partial sums) is allocated and freed on
 * `stream` inside the call; returns after synchronizing `stream`.
 */
int ubqp_penalized_eval(const void* Q, const void* b, const void* p, const void* x, int64_t n,
                        int64_t batch, int dtype, void* h_out, void* g_out, void* stream);

/*
 * ubqp_penalized_vjp - backward of ubqp_penalized_eval (the vector-Jacobian product of h
 * with respect to x, p and b), for `batch` points and the output gradient grad_h:
 *     gx[r][i] = grad_h[r] g[r][i],  gp[i] = sum_r grad_h[r] (x_ri - x_ri^2),
 *     gb[i] = sum_r grad_h[r] x_ri
 * (h is linear in p and b, so these are exact derivatives).  All pointers are DEVICE
 * memory of element type dtype: x and g (the g_out of the forward call) batch x n,
 * grad_h batch; gx_out batch x n, gp_out n and gb_out n, each may be NULL (g may be NULL
 * when gx_out is).  The sums over r run in FP64 in order r = 0, 1, ...  Allocates nothing;
 * returns after synchronizing `stream`.
 */
int ubqp_penalized_vjp(const void* x, const void* g, const void* grad_h, int64_t n, int64_t batch, int dtype,
                       void* gx_out, void* gp_out, void* gb_out, void* stream);

/*
 * ubqp_penalized_eval_noalloc - the computation of ubqp_penalized_eval (h and grad h of
 * problem (p) for `batch` points, same arguments, same kernel, same work partition) without
 * any device allocation, for callers that cannot call cudaMalloc/cudaFree: code that owns
 * all device memory through its own pool or a fixed memory budget, and code that cannot
 * afford the device-wide synchronization those calls may cause.  The paper has no
 * counterpart; this is an interface variant of this library.
 *   Scratch: a static device array of UBQP_NOALLOC_SCRATCH_BYTES that every GPU loading the
 *   library holds until the process exits.  Limits: batch <= 256, n * element size <=
 *   200 KiB, and batch * ceil(n / rows per item) <= 16384 work items (rows per item as in
 *   ubqp_penalized_eval, at most 256); larger requests return UBQP_EINVAL with the limit
 *   named in ubqp_last_error().
 *   The array's device address is resolved (cudaGetSymbolAddress) on the first call in each
 *   CUDA context, so make that first call before any stream capture in that context; a new
 *   context (after a device reset) gets its own first call.
 *   All calls share the array and it keeps the last call's contents (each call rewrites
 *   what it reads); calls that overlap on the GPU (other streams, other host threads) race.
 *   All pointers are device memory.  The call ends with cudaStreamSynchronize(stream), so
 *   it cannot be called on a stream that is being captured.
 */
#define UBQP_NOALLOC_SCRATCH_BYTES 2310400
int ubqp_penalized_eval_noalloc(const void* Q, const void* b, const void* p, const void* x, int64_t n,
                                int64_t batch, int dtype, void* h_out, void* g_out, void* stream);

/*
 * ubqp_inner_run - test entry: Alg. 2 (or Alg. 1 when o->method = UBQP_PPA) on the
 * subproblem (p1) with a GIVEN reformulated matrix Qp = Q' (n x n, diagonal included),
 * bp = b', penalty p and start x0 (all FP64, host or device), on the FP32 GPU path.
 *   trace_len  iterates to record; trace_x (trace_len x n) receives x_k and trace_alpha
 *              (trace_len) the step used at iteration k (host or device; may be NULL).
 *   x_out (n), steps_out, exit_out (0 KKT test met, 1 iteration cap, 2 zero step).
 */
int ubqp_inner_run(const double* Qp, const double* bp, const double* p, const double* x0,
                   int64_t n, const ubqp_opts* o, int32_t trace_len, double* trace_x,
                   double* trace_alpha, double* x_out, int32_t* steps_out, int32_t* exit_out);

/*
 * ubqp_penalty_probe - test entry: one penalty step of Sec. 3.4 on the GPU for a given
 * state (Qp, bp, p, x as in ubqp_inner_run): lambda_min of Z^-1/2 Qbar_II Z^-1/2 by the
 * device eigen-solver, the step alpha (Eq. (eq:alpha1) with the resolution floor, no
 * previous floor steps), |I| and the eigen-solver iterations.  Outputs are host memory.
 * o->precision selects the matrix-vector products: UBQP_FP32 (the FP32 GEMV kernels) or a
 * tensor-core precision (the BF16 contraction of the batched path; the off-diagonal of Qp
 * must then be exact in BF16, else UBQP_ENOTSUP).
 */
int ubqp_penalty_probe(const double* Qp, const double* bp, const double* p, const double* x,
                       int64_t n, const ubqp_opts* o, double* lambda_out, double* alpha_out,
                       int32_t* n_active_out, int32_t* iters_out);

/*
 * ubqp_initial_point - test entry: the device initialization of Sec. 3.5 for one instance
 * (perturbation mu, host/device n x n or NULL; reformulation; x^0 of Eq. (gamma) by
 * Jacobi sweeps on the FP32 path).  x0_out (n) and gamma_out (n, may be NULL), host or
 * device, FP64.
 */
int ubqp_initial_point(const double* Q, const double* b, const double* mu, int64_t n,
                       const ubqp_opts* o, double* x0_out, double* gamma_out);

/*
 * ubqp_profile_timeline - the per-tick record of the last call on this thread that ran
 * with profile_kernels = 2: the phase-A duration of every tick (ms, CUDA events) and the
 * algorithmic bytes (FP32 path) or flops (tensor-core path) that tick processed.  Copies up
 * to `cap` entries into host arrays (either may be NULL) and returns the number recorded.
 */
int64_t ubqp_profile_timeline(float* ms_out, int64_t* work_out, int64_t cap);

/*
 * ubqp_tc_matmul_probe - test entry: the tensor-core contraction of the batched path on
 * its own, D = A (B_hi + B_lo)^T with FP32 accumulation, returned raw.
 *   A n x n, B_hi and B_lo (B_lo may be NULL) R x n, all BF16 bit patterns in HOST memory,
 *   row-major; D_out R x n FP32 host memory (row r = lane r).  cluster: CTAs splitting K
 *   (1..8), 0 = picked by the library, -1 = the persistent kernel of many-tile launches
 *   (no split-K).  1 <= n <= 32768, 1 <= R <= 1024.
 */
int ubqp_tc_matmul_probe(const uint16_t* A, const uint16_t* B_hi, const uint16_t* B_lo, int64_t n, int64_t R,
                         int32_t cluster, float* D_out);

#ifdef __cplusplus
}
#endif
#endif /* UBQP_H */
