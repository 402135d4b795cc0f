// Internal device-side definitions of the vectorized PSDP solver (arXiv 2408.04875).
//
// Execution model.  Every (instance, start) pair is a *lane* that runs Alg. 3 as a
// small state machine.  All lanes advance together in *ticks*; one tick is
//   phase A  one matvec per active lane,  v = Q_off u  (FP32 GEMV kernel, or the
//            tcgen05 BF16 contraction when the starts of one instance are batched),
//            followed by a per-row epilogue that depends on the lane's phase and
//            writes per-block partial sums;
//   phase B  one CTA per lane: reduce the partials, take the lane's scalar decision
//            (BB step, KKT test, eigen-solver step, penalty step, ...), apply the
//            element-wise update and write the next matvec input u.
// Every step of the paper that touches Q (gradient Eq. (x2)/(x1), the matvecs of the
// lambda_min solver of Eq. (eq:alpha), the Jacobi sweeps for Eq. (gamma), the exact
// evaluation of rounded points) is one tick; everything else is element-wise.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ubqp {

// ---------------------------------------------------------------------------------
// lane phases
enum Phase : int32_t {
    PH_DONE = 0,
    PH_JACOBI = 1,    // x^0 of Eq. (gamma): x <- (-b' - 2 Q_off x) / (2 d)
    PH_EVAL = 2,      // exact f of the rounded iterate, outer stopping test of Alg. 3
    PH_LOB_INIT = 3,  // first matvec of the lambda_min solver (A x_0)
    PH_LOB = 4,       // one LOBPCG iteration for lambda_min of Z^-1/2 Qbar_II Z^-1/2
    PH_INNER = 5,     // one iteration of Alg. 2 (PABB) or Alg. 1 (PPA)
    PH_GRAD = 6,      // stand-alone h and gradient (penalized_eval)
};

enum LaneMode : int32_t { MODE_GEMV = 0, MODE_TC = 1, MODE_GRAD = 2 };

// stop hooks used by the test entry points
enum StopAfter : int32_t { STOP_INNER = 1, STOP_LOB = 2, STOP_JACOBI = 4 };

// per-lane FP32 vectors, each `ld` long
enum Vec : int32_t {
    V_X = 0,   // current iterate x
    V_XPREV,   // previous iterate (Alg. 2, s = x_k - x_{k-1})
    V_G,       // gradient g_k (phase A writes it in place of g_{k-1})
    V_P,       // penalty p (Eq. (pp1))
    V_DMP,     // d - p  (diagonal of Qbar)
    V_BBAR,    // b' + p
    V_D,       // z^-1/2 on I_alpha, 0 elsewhere (scaling of Eq. (eq:alpha))
    V_T,       // Jacobi preconditioner of the eigen-solver, 1/|A_ii| = z_i/|d_i - p_i|
    V_LX,      // eigen-solver iterate
    V_LAX,     // A * LX
    V_LP,      // eigen-solver previous direction
    V_LAP,     // A * LP
    V_LW,      // preconditioned residual
    V_W,       // phase-A output (A w, or the Jacobi update)
    V_U,       // next matvec input (FP32 GEMV lanes)
    NVEC
};

// one per (lane, phase-A block): 128 bytes
struct __align__(16) Partial {
    float2 s[12];   // compensated sums (hi, lo)
    float m[6];     // maxima (all values >= 0)
    double f;       // FP64 sum (objective of a rounded point / h of penalized_eval)
};
static_assert(sizeof(Partial) == 128, "Partial must stay 128 bytes");

// mutable scalar state of one lane, owned by its phase-B CTA
struct __align__(16) LaneState {
    int32_t phase;
    int32_t k;          // inner iteration within the current subproblem
    int32_t s;          // outer step = subproblems solved so far
    int32_t it;         // Jacobi sweep / eigen-solver iteration
    int32_t consec_fb;  // consecutive penalty steps that used the resolution floor
    int32_t has_p;      // eigen-solver has a previous direction
    int32_t status;     // 0 ok, 1 outer cap
    int32_t last_exit;  // exit code of the last subproblem (0 KKT, 1 cap, 2 zero step)
    float alpha;        // current BB step (Eq. (bb1))
    float rho;          // rho of Eq. (cret) for the current p
    float lam;          // Ritz value of the eigen-solver
    float pen_alpha;    // last penalty step
    double best_f;      // best exact objective of a rounded iterate
    int32_t best_s;
    int32_t n_active;   // |I_alpha| at the last evaluation
    int64_t inner_iters;
    int64_t inner_steps;
    int64_t lob_iters;
    int64_t jac_iters;
    int64_t floor_steps;
    int64_t updates;    // steps (updates) this lane has taken
};

// static description of one lane (written by the host, read-only on the device)
struct LaneDev {
    int32_t n;          // problem size
    int32_t ld;         // padded length of every vector / row stride of Q_off
    int32_t mode;       // LaneMode
    int32_t nblk;       // phase-A blocks (partials) of this lane
    int32_t method;     // 0 PABB, 1 PPA
    int32_t stop_after; // StopAfter bits
    int32_t restart;    // index of this start within its instance (TC operand row)
    int32_t trace_len;
    const float* Qoff;     // GEMV lanes: n x ld FP32, off-diagonal of Q' (zero diagonal)
    const float2* Qeval;   // GEMV lanes: n x ld, the original Q as FP32 (hi, lo) pairs
    const float* d;        // diag(Q')
    const float* bprime;   // b - gamma
    const float* tsum;     // diag(Q') + b' = (Q + mu)_ii + b_i, formed in FP64
    const float* oabs;     // sum_{j != i} |Q'_ij|
    const float* rabs;     // sum_j |Q'_ij|
    const double* borig;   // original b (GEMV eval), may be null
    const double* qdb;     // Q_ii + b_i of the original data (TC eval)
    float* vec;            // NVEC * ld floats
    uint8_t* best_x;       // ld bytes
    Partial* part;         // nblk partials
    LaneState* st;
    unsigned int* counter; // phase-A blocks of the current tick that have finished
    __nv_bfloat16* u_hi;   // TC lanes: this lane's row of the packed B operand
    __nv_bfloat16* u_lo;
    float* trace_x;        // test hook: trace_len x n
    float* trace_alpha;
    float qmax_off;        // max_{i != j} |Q'_ij|
    float rabs_max;        // max_i rabs_i
    // gradient lanes (penalized_eval)
    const void* gQ;
    const void* gb;
    const void* gp;
    const void* gx;
    void* gg;
    int32_t gld;
    int32_t spwps;         // sliced storage: warps per 32-row slice (8 / slices per item)
    int32_t* nt_active;    // TC lanes: unfinished lanes of this lane's N tile (decremented
                           // by the update that finishes the lane), else null
    // sliced row storage of Q'_off (GEMV lanes, sparse data), or null: entry spo[s] + 32 k + r
    // of slice s is the k-th stored entry of row 32 s + r (value spv, column spc)
    const float* spv;
    const uint16_t* spc;
    const int64_t* spo;
};

// solver constants (kernel parameter)
struct Params {
    int32_t max_outer, max_inner, lob_max, jac_max;
    float tol_inner, tol_outer, eta, alpha_min, alpha_max, tau_z, eps_hp_rel, lambda_floor_rel;
    float lob_tol, jac_tol;
    int64_t* hist;       // UBQP_HIST_BINS counters (may be null)
    unsigned long long* bytes;  // algorithmic bytes read by phase A (may be null)
};

// ---------------------------------------------------------------------------------
// compensated (Neumaier / TwoSum) FP32 summation

// Knuth's TwoSum: s + e == a + b exactly.  The _rn intrinsics keep the compiler from
// contracting a product feeding `b` into an FMA, which would break the identity.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void csum_add(float2& acc, float v)
{
    float s, e;
    two_sum(acc.x, v, s, e);
    acc.x = s;
    acc.y += e;
}

__device__ __forceinline__ float2 csum_merge(float2 a, float2 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    return make_float2(s, a.y + b.y + e);
}

__device__ __forceinline__ float2 csum_shfl_reduce(float2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 w;
        w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = csum_merge(v, w);
    }
    return v;
}

__device__ __forceinline__ float max_shfl_reduce(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double dsum_shfl_reduce(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// per-thread accumulator of one phase-A block
struct Acc {
    float2 s[12];
    float m[6];
    double f;
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int t = 0; t < 12; ++t) s[t] = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 6; ++t) m[t] = 0.f;
        f = 0.0;
    }
};

// how many compensated sums / maxima each phase uses (keeps reductions short)
__device__ __forceinline__ int phase_nsum(int ph)
{
    switch (ph) {
    case PH_INNER: return 3;
    case PH_EVAL: return 1;
    case PH_LOB_INIT: return 2;
    case PH_LOB: return 12;
    default: return 0;
    }
}
constexpr int phase_nsum_inner = 3, phase_nmax_inner = 4;   // phase_nsum / phase_nmax of PH_INNER
__device__ __forceinline__ int phase_nmax(int ph)
{
    switch (ph) {
    case PH_INNER: return 4;
    case PH_EVAL: return 3;
    case PH_JACOBI: return 2;
    default: return 0;
    }
}

// ---------------------------------------------------------------------------------
// Per-row epilogue of phase A.  Row i of lane L received v = (Q_off u)_i (for EVAL on
// GEMV lanes: (Q_orig u)_i in FP64).  k is the inner iteration of the lane.

__device__ __forceinline__ void row_epilogue(const LaneDev& L, int ph, int k, int i, double vd,
                                             Acc& a, float tau_z)
{
    float* vec = L.vec;
    const int ld = L.ld;
    float v = (float)vd;
    switch (ph) {
    case PH_INNER: {
        // g = 2 Qbar x + bbar = 2 Q_off x + 2 (d - p) x + (b' + p)   (Alg. 2: g^k), evaluated as
        // 2 Q_off x + (d - p)(2x - 1) + (d + b'): the two gamma-sized terms of the diagonal
        // part cancel analytically instead of in FP32 (2x - 1 is exact for x in [1/4, 1]).
        float x = vec[V_X * ld + i];
        float dmp = vec[V_DMP * ld + i];
        float bb = vec[V_BBAR * ld + i];
        float g = fmaf(dmp, 2.f * x - 1.f, fmaf(2.f, v, L.tsum[i]));
        if (k >= 1) {  // Eq. (bb1): s_{k-1} = x_k - x_{k-1}, y_{k-1} = g_k - g_{k-1}
            float s = x - vec[V_XPREV * ld + i];
            float y = g - vec[V_G * ld + i];
            csum_add(a.s[0], s * s);
            csum_add(a.s[1], s * y);
            csum_add(a.s[2], y * y);
        } else {      // quantities of rho (Eq. (cret)) and ||Qbar||_inf for alpha_0
            a.m[1] = fmaxf(a.m[1], fabsf(dmp));
            a.m[2] = fmaxf(a.m[2], fabsf(bb));
            a.m[3] = fmaxf(a.m[3], L.oabs[i] + fabsf(dmp));
        }
        vec[V_G * ld + i] = g;
        // Eq. (cret): |g| on I, max(-g,0) on J (x = 0), max(g,0) on K (x = 1)
        float viol = (x > 0.f && x < 1.f) ? fabsf(g) : (x <= 0.f ? fmaxf(-g, 0.f) : fmaxf(g, 0.f));
        a.m[0] = fmaxf(a.m[0], viol);
        break;
    }
    case PH_EVAL: {
        float x = vec[V_X * ld + i];
        if (x > 0.5f) {
            double lin = (L.mode == MODE_TC) ? L.qdb[i] : (L.borig ? L.borig[i] : 0.0);
            a.f += vd + lin;
        }
        a.m[0] = fmaxf(a.m[0], fminf(x, 1.f - x));
        float z = x - x * x;
        if (z > tau_z) a.s[0].x += 1.f;
        a.m[1] = fmaxf(a.m[1], fabsf(vec[V_DMP * ld + i]));
        a.m[2] = fmaxf(a.m[2], fabsf(vec[V_BBAR * ld + i]));
        break;
    }
    case PH_LOB_INIT:
    case PH_LOB: {
        // A = Z^-1/2 Qbar_II Z^-1/2 applied to w:  (A w)_i = D_i ((Q_off u)_i + (d_i - p_i) u_i),
        // u = D w (zero outside I_alpha)
        float Dz = vec[V_D * ld + i];
        float w = (ph == PH_LOB_INIT) ? vec[V_LX * ld + i] : vec[V_LW * ld + i];
        float aw = 0.f;
        if (Dz != 0.f) aw = Dz * fmaf(vec[V_DMP * ld + i], Dz * w, v);
        vec[V_W * ld + i] = aw;
        if (ph == PH_LOB_INIT) {
            csum_add(a.s[0], w * aw);
            csum_add(a.s[1], w * w);
        } else {
            float x = vec[V_LX * ld + i], ax = vec[V_LAX * ld + i];
            float p = vec[V_LP * ld + i], ap = vec[V_LAP * ld + i];
            csum_add(a.s[0], x * ax);
            csum_add(a.s[1], x * aw);
            csum_add(a.s[2], x * ap);
            csum_add(a.s[3], w * aw);
            csum_add(a.s[4], w * ap);
            csum_add(a.s[5], p * ap);
            csum_add(a.s[6], x * x);
            csum_add(a.s[7], x * w);
            csum_add(a.s[8], x * p);
            csum_add(a.s[9], w * w);
            csum_add(a.s[10], w * p);
            csum_add(a.s[11], p * p);
        }
        break;
    }
    case PH_JACOBI: {
        // Eq. (gamma): 2 (Q_off + Diag d) x = -b'  ->  x_i = (-b'_i - 2 (Q_off x)_i) / (2 d_i)
        float xn = (-L.bprime[i] - 2.f * v) / (2.f * L.d[i]);
        a.m[0] = fmaxf(a.m[0], fabsf(xn - vec[V_X * ld + i]));
        a.m[1] = fmaxf(a.m[1], fabsf(xn));
        vec[V_W * ld + i] = xn;
        break;
    }
    default: break;
    }
}

// ---------------------------------------------------------------------------------
// Block-wide reduction of Acc into one Partial (blockDim.x threads, <= 1024)

// The warp's butterfly reduction of a phase's sums (compensated), maxima and FP64 sum: for
// every quantity the shuffles xor 16, 8, 4, 2, 1 in that order.  The inner step (3 sums, 4
// maxima) and the eigen-solver step (12 sums, six at a time) run their quantities level by
// level so that the chains overlap; the result of each quantity is the same either way.
__device__ __forceinline__ void acc_shfl_reduce(Acc& a, int ph, bool has_f)
{
    static_assert(phase_nsum_inner == 3 && phase_nmax_inner == 4, "inner-step partials");
    if (ph == PH_INNER) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 w[3];
            float wm[4];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                w[t].x = __shfl_xor_sync(0xffffffffu, a.s[t].x, o);
                w[t].y = __shfl_xor_sync(0xffffffffu, a.s[t].y, o);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) wm[t] = __shfl_xor_sync(0xffffffffu, a.m[t], o);
#pragma unroll
            for (int t = 0; t < 3; ++t) a.s[t] = csum_merge(a.s[t], w[t]);
#pragma unroll
            for (int t = 0; t < 4; ++t) a.m[t] = fmaxf(a.m[t], wm[t]);
        }
    } else if (ph == PH_LOB) {
        // six sums at a time (registers)
#pragma unroll
        for (int h = 0; h < 12; h += 6)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float2 w[6];
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    w[t].x = __shfl_xor_sync(0xffffffffu, a.s[h + t].x, o);
                    w[t].y = __shfl_xor_sync(0xffffffffu, a.s[h + t].y, o);
                }
#pragma unroll
                for (int t = 0; t < 6; ++t) a.s[h + t] = csum_merge(a.s[h + t], w[t]);
            }
    } else {
        const int ns = phase_nsum(ph), nm = phase_nmax(ph);
#pragma unroll
        for (int t = 0; t < 12; ++t)
            if (t < ns) a.s[t] = csum_shfl_reduce(a.s[t]);
#pragma unroll
        for (int t = 0; t < 6; ++t)
            if (t < nm) a.m[t] = max_shfl_reduce(a.m[t]);
    }
    if (has_f) a.f = dsum_shfl_reduce(a.f);
}

template <int NWARP>
__device__ __forceinline__ void block_reduce_write(Acc& a, int ph, Partial* out, bool has_f)
{
    __shared__ float2 sh_s[NWARP][12];
    __shared__ float sh_m[NWARP][6];
    __shared__ double sh_f[NWARP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ns = phase_nsum(ph), nm = phase_nmax(ph);
    // (the plain per-quantity butterflies: this function is inlined at many call sites, and the
    // level-by-level variants there made the single-lane kernel measurably slower)
#pragma unroll
    for (int t = 0; t < 12; ++t)
        if (t < ns) a.s[t] = csum_shfl_reduce(a.s[t]);
#pragma unroll
    for (int t = 0; t < 6; ++t)
        if (t < nm) a.m[t] = max_shfl_reduce(a.m[t]);
    if (has_f) a.f = dsum_shfl_reduce(a.f);
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < 12; ++t)
            if (t < ns) sh_s[warp][t] = a.s[t];
#pragma unroll
        for (int t = 0; t < 6; ++t)
            if (t < nm) sh_m[warp][t] = a.m[t];
        sh_f[warp] = has_f ? a.f : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial P;
        for (int t = 0; t < 12; ++t) P.s[t] = make_float2(0.f, 0.f);
        for (int t = 0; t < 6; ++t) P.m[t] = 0.f;
        P.f = 0.0;
        for (int w = 0; w < NWARP; ++w) {
            for (int t = 0; t < ns; ++t) P.s[t] = csum_merge(P.s[t], sh_s[w][t]);
            for (int t = 0; t < nm; ++t) P.m[t] = fmaxf(P.m[t], sh_m[w][t]);
            P.f += sh_f[w];
        }
        *out = P;
    }
}

// ---------------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)

struct TickArgs {
    const LaneDev* lanes;
    const int2* items;     // GEMV phase-A work items: (lane, block)
    int32_t nitems;
    int32_t rows_per_item;
    int32_t nlanes;
    int32_t max_ld;        // widest lane (shared-memory size of the GEMV kernel)
    int32_t fused;         // GEMV lanes: the last phase-A CTA of a lane runs its update
    int32_t grid;          // persistent GEMV grid size
    int32_t* active_count; // incremented by every lane still active after this tick
    int32_t* work;         // GEMV work queue head (reset by the last CTA of a tick)
    int32_t* done;         // CTAs of the tick that have left the queue
    Params P;
};

cudaError_t prepare_phase_a_gemv(int max_ld);
int gemv_grid(int max_ld, int nitems);
cudaError_t launch_phase_a_gemv_f32(const TickArgs& a, cudaStream_t s);
cudaError_t launch_phase_a_grad(const TickArgs& a, int dtype, int64_t n, cudaStream_t s);
constexpr int kSymT = 128;   // tile edge of the symmetric storage
constexpr int kSymGroup = 2; // tiles per first-stage ring entry

// one lane's symmetric storage (persistent lane loop): the packed upper-triangle tiles of
// its instance, its partial vectors (nb x ld floats) and the counter of its tiles this step
struct SymLane {
    const float* Qsym;
    float* pbuf;
    unsigned int* counter;
    int32_t nb;                 // row blocks of kSymT rows
    int32_t ntiles;             // nb (nb + 1) / 2
    int32_t ngroups;            // first-stage entries: ceil(ntiles / kSymGroup)
};

// seeded ring slots of one lane: its current step is either a tile step (ngroups entries) or
// an evaluation step (nb row-block entries), so it gets the larger count and the seed skips
// the slots its step does not use
inline int sym_slots(const SymLane& S) { return S.ngroups > S.nb ? S.ngroups : S.nb; }

// persistent lane loop (GEMV lanes): a ring of (lane, row block) entries shared by all CTAs
struct LoopArgs {
    const LaneDev* lanes;
    const int2* items;          // every lane's blocks, largest lanes first (seeding order)
    int32_t nitems;
    int32_t nlanes;
    int32_t rows_per_item;
    int32_t max_ld;
    int32_t budget;             // steps each lane may take in one launch
    int32_t grid;               // CTAs of the loop kernel
    unsigned long long* ring;   // cap slots: (sequence << 32) | (lane << 16) | block
    unsigned long long cap;     // power of two >= 2 (nitems + grid)
    unsigned long long* head;   // positions popped
    unsigned long long* tail;   // positions pushed
    int32_t* running;           // lanes that may still push in this launch
    int32_t* active_after;      // lanes unfinished when the launch ends
    int32_t* err;               // set when a bounded wait runs out
    int32_t* budget_left;       // per lane
    const SymLane* sym;         // per lane, or null: dense rows
    unsigned long long wait_ns; // limit of one wait for a ring slot
    Params P;
};

// FP32 lanes as one persistent cooperative launch (solo.cu): the CTAs form groups, and each
// group runs its lanes one after another, every lane on all CTAs of its group
struct SoloArgs {
    const LaneDev* lane;        // the lanes
    const int32_t* glanes;      // lane indices, group after group (null: lane 0 alone)
    const int32_t* gfirst;      // group g's lanes: glanes[gfirst[g] .. gfirst[g+1])
    const int32_t* gcta;        // group g's CTAs: gcta[g] .. gcta[g+1]-1 (null: one group)
    int32_t ngroups;
    int32_t rows_per_item;
    int32_t budget;             // steps each group may take in this launch
    int32_t grid;
    unsigned* bar;              // per group (stride kSoloBarStride words): a 64-bit arrival counter
    int32_t* err;               // set when a bounded wait runs out
    int32_t* active_after;      // lanes unfinished at the end of the launch (the caller zeroes it)
    unsigned long long wait_ns; // limit of one barrier wait
    int32_t fast;               // Alg. 2 steps with one barrier (whole x_k in every CTA)
    int32_t one_ok;             // shared memory holds the one-CTA state (6 vectors)
    Params P;
};
constexpr int kSoloBarStride = 32;   // unsigned per group barrier (128 bytes)
constexpr int kSoloMaxSl = 5;        // most 32-row slices a CTA of the lane groups computes per step
void solo_shape(int n, int rows_per_item, int sms, int* grid, int* rb, int* nblk);
size_t solo_smem(int ld, bool one);
cudaError_t prepare_solo(int ld, bool one);
int solo_ctas_per_sm(int ld, bool one);
cudaError_t launch_solo(const SoloArgs& a, int ld, cudaStream_t s);

cudaError_t prepare_lane_loop(int max_ld);
int lane_loop_grid(int max_ld);
cudaError_t launch_lane_loop(const LoopArgs& a, cudaStream_t s);   // seed + loop kernels
cudaError_t launch_phase_b(const TickArgs& a, int32_t* active_count, cudaStream_t s);
cudaError_t launch_grad_reduce(const LaneDev* lanes, int nlanes, void* h_out, int dtype,
                               cudaStream_t s);
cudaError_t launch_grad_setup(LaneDev* lanes, int2* items, int32_t* queue, Partial* part, const void* Q, const void* b,
                              const void* p, const void* x, void* g, int n, int batch, int nblk, int es, cudaStream_t s);
cudaError_t launch_penalized_vjp(const void* x, const void* g, const void* go, int64_t n, int64_t batch, int dtype,
                                 void* gx, void* gp, void* gb, cudaStream_t s);

// the calling thread's last-error text (ubqp_last_error), shared by every entry point
void set_error(const char* fmt, ...);
void clear_error();

}  // namespace ubqp
