// Phase B: one CTA per lane.  Reduces the lane's phase-A partials, takes the scalar
// decision of the lane's phase and applies the element-wise update:
//   INNER   Alg. 2: KKT test of Eq. (cret), alternating BB step of Eq. (bb1) with the
//           safeguards listed below, projected step of Eq. (x2); or Alg. 1: the
//           per-coordinate step of Eq. (x1) with H_p of Sec. 3.1.
//   EVAL    exact objective of the rounded iterate, best-so-far, outer test of Alg. 3.
//   LOB*    one LOBPCG iteration (Jacobi preconditioned, 3x3 Rayleigh-Ritz) for
//           lambda_min of Z^-1/2 Qbar_II Z^-1/2 (Lemma 3.1); on convergence the penalty
//           update p += alpha z of Eq. (pp1) with alpha of Eq. (eq:alpha1).
//   JACOBI  one sweep for x^0 of Eq. (gamma).
// Safeguards of the BB step (the paper states none): alpha_0 = 1/(2 ||Qbar||_inf);
// s^T y <= 0 or a non-finite ratio keeps the previous step; clamp to
// [alpha_min, alpha_max]; s = 0 stops the subproblem.
#pragma once
#include "ubqp_internal.cuh"

namespace ubqp {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;

enum Action : int32_t {
    A_COPY_W_X = 1 << 0,
    A_SAVE_BEST = 1 << 1,
    A_LOB_SETUP = 1 << 2,
    A_LOB_NORM = 1 << 3,
    A_LOB_UPDATE = 1 << 4,
    A_RESID = 1 << 5,
    A_PENALTY = 1 << 6,
    A_STEP_PABB = 1 << 7,
    A_STEP_PPA = 1 << 8,
    A_TRACE = 1 << 9,
};
enum USource : int32_t { U_NONE = 0, U_X, U_ROUND, U_DLX, U_DLW };

struct Decision {
    int32_t act;
    int32_t usrc;
    float alpha;   // BB step / penalty step
    float lam;     // Ritz value (residual)
    float c0, cx, cw, cp;
    float eps_hp;
    int32_t trace_k;
};

// deterministic start vector of the eigen-solver: uniform in (-1, 1) from a hash of i
__device__ __forceinline__ float start_component(int i)
{
    uint32_t h = (uint32_t)i * 0x9E3779B1u + 0x7F4A7C15u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return ((float)(h >> 8) + 0.5f) * (2.0f / 16777216.0f) - 1.0f;
}

// 1/sqrt(v): the hardware reciprocal square root on the device; the host form (the two
// functions below also compile for the host, where the tests pin them) divides by sqrtf
__host__ __device__ __forceinline__ float rr_rsqrt(float v)
{
#ifdef __CUDA_ARCH__
    return rsqrtf(v);
#else
    return 1.0f / sqrtf(v);
#endif
}

// smallest eigenpair of a symmetric k x k matrix (k <= 3) by cyclic Jacobi rotations.
// FP32 throughout: FP64 runs at a small fraction of the FP32 rate on this part, and the
// preconditioned basis keeps the 3 x 3 Gram matrices well scaled.  Every loop runs over the
// full 3 x 3 with the entries outside k x k masked, so that all indices are compile-time
// constants and the matrices stay in registers (the operations and their order are those
// of the k x k loops).
__host__ __device__ __forceinline__ void small_sym_eig_min(int k, float (&M)[3][3], float& lam, float (&v)[3])
{
    float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
    for (int sweep = 0; sweep < 8; ++sweep) {
        float off = 0.f, dia = 0.f;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            if (p >= k) break;
            dia += M[p][p] * M[p][p];
#pragma unroll
            for (int q = p + 1; q < 3; ++q)
                if (q < k) off += M[p][q] * M[p][q];
        }
        if (off <= 1e-14f * dia) break;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = p + 1; q < 3; ++q) {
                if (q >= k || M[p][q] == 0.f) continue;
                float theta = (M[q][q] - M[p][p]) / (2.f * M[p][q]);
                float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                float c = rr_rsqrt(t * t + 1.f), sn = t * c;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (r >= k) break;
                    float mrp = M[r][p], mrq = M[r][q];
                    M[r][p] = c * mrp - sn * mrq;
                    M[r][q] = sn * mrp + c * mrq;
                }
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (r >= k) break;
                    float mpr = M[p][r], mqr = M[q][r];
                    M[p][r] = c * mpr - sn * mqr;
                    M[q][r] = sn * mpr + c * mqr;
                }
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (r >= k) break;
                    float vrp = V[r][p], vrq = V[r][q];
                    V[r][p] = c * vrp - sn * vrq;
                    V[r][q] = sn * vrp + c * vrq;
                }
            }
    }
    int j = 0;
    lam = M[0][0];
    if (k > 1 && M[1][1] < lam) { j = 1; lam = M[1][1]; }
    if (k > 2 && M[2][2] < lam) { j = 2; lam = M[2][2]; }
#pragma unroll
    for (int r = 0; r < 3; ++r) v[r] = r < k ? (j == 0 ? V[r][0] : (j == 1 ? V[r][1] : V[r][2])) : 0.f;
}

// Rayleigh-Ritz on span{x, w, p} (p only when has_p), FP32.  Returns false on breakdown.
// Gram entries: ga = (xAx, xAw, xAp, wAw, wAp, pAp), gb = (xx, xw, xp, ww, wp, pp).
// Loops as in small_sym_eig_min: full 3 x 3, masked to k x k.  Not inlined: its registers are
// needed only for the eigen-solver's decision, not in the kernels' hot loops.
static __host__ __device__ __noinline__ bool rayleigh_ritz(const float (&ga)[6], const float (&gb)[6], bool has_p, float& lam,
                                              float (&c)[3])
{
    const float A[3][3] = {{ga[0], ga[1], ga[2]}, {ga[1], ga[3], ga[4]}, {ga[2], ga[4], ga[5]}};
    const float B[3][3] = {{gb[0], gb[1], gb[2]}, {gb[1], gb[3], gb[4]}, {gb[2], gb[4], gb[5]}};
    int k = has_p ? 3 : 2;
    if (!(B[0][0] > 0.f)) return false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (k < 2) return false;
        float sc[3] = {0.f, 0.f, 0.f};
        bool bad = false;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t >= k) break;
            if (!(B[t][t] > 0.f)) { bad = true; break; }
            sc[t] = rr_rsqrt(B[t][t]);
        }
        if (bad) { k -= 1; continue; }
        float As[3][3], Bs[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                As[r][q] = (r < k && q < k) ? A[r][q] * sc[r] * sc[q] : 0.f;
                Bs[r][q] = (r < k && q < k) ? B[r][q] * sc[r] * sc[q] : 0.f;
            }
        // Cholesky Bs = L L^T; a pivot below 1e-3 (unit diagonal) means a nearly dependent
        // basis in FP32: drop the last direction and retry
        float Lc[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= k || bad) break;
            float sd = Bs[j][j];
#pragma unroll
            for (int t = 0; t < j; ++t) sd -= Lc[j][t] * Lc[j][t];
            if (!(sd > 1e-3f)) { bad = true; break; }
            Lc[j][j] = sqrtf(sd);
#pragma unroll
            for (int i = j + 1; i < 3; ++i) {
                if (i >= k) break;
                float u = Bs[i][j];
#pragma unroll
                for (int t = 0; t < j; ++t) u -= Lc[i][t] * Lc[j][t];
                Lc[i][j] = u / Lc[j][j];
            }
        }
        if (bad) { k -= 1; continue; }
        float Li[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= k) break;
            Li[j][j] = 1.f / Lc[j][j];
#pragma unroll
            for (int i = j + 1; i < 3; ++i) {
                if (i >= k) break;
                float u = 0.f;
#pragma unroll
                for (int t = j; t < i; ++t) u -= Lc[i][t] * Li[t][j];
                Li[i][j] = u / Lc[i][i];
            }
        }
        float M[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float u = 0.f;
                if (r < k && q < k)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (a >= k) break;
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            if (b >= k) break;
                            u += Li[r][a] * As[a][b] * Li[q][b];
                        }
                    }
                M[r][q] = u;
            }
        float v[3];
        small_sym_eig_min(k, M, lam, v);
#pragma unroll
        for (int r = 0; r < 3; ++r) {  // c = sc * L^-T v
            float u = 0.f;
#pragma unroll
            for (int a = r; a < 3; ++a) {
                if (a >= k) break;
                u += Li[a][r] * v[a];
            }
            c[r] = r < k ? u * sc[r] : 0.f;
        }
        return isfinite(lam);
    }
    return false;
}

__device__ __forceinline__ float csum_value(float2 v) { return v.x + v.y; }

// Scalar decision of one lane (thread 0).  S is the lane state (shared memory).
static __device__ void decide(const LaneDev& L, LaneState& S, const Partial& R, const Params& P, Decision& D)
{
    D.act = 0;
    D.usrc = U_NONE;
    D.alpha = 0.f;
    D.lam = 0.f;
    D.c0 = D.cx = D.cw = D.cp = 0.f;
    D.eps_hp = P.eps_hp_rel * fmaxf(1.f, L.rabs_max);
    D.trace_k = -1;
    switch (S.phase) {
    case PH_JACOBI: {
        S.it += 1;
        S.jac_iters += 1;
        D.act |= A_COPY_W_X;
        bool conv = R.m[0] <= P.jac_tol * fmaxf(R.m[1], 1e-30f) || S.it >= P.jac_max;
        if (!conv) { D.usrc = U_X; break; }
        S.it = 0;
        if (L.stop_after & STOP_JACOBI) { S.phase = PH_DONE; break; }
        S.phase = PH_EVAL;
        D.usrc = U_ROUND;
        break;
    }
    case PH_EVAL: {
        double f = R.f;
        float bin = R.m[0];
        int active = (int)(R.s[0].x + R.s[0].y);
        S.rho = fmaxf(fmaxf(1.f, 2.f * L.qmax_off), fmaxf(2.f * R.m[1], R.m[2]));
        S.n_active = active;
        if (f < S.best_f) {
            S.best_f = f;
            S.best_s = S.s;
            D.act |= A_SAVE_BEST;
        }
        if (bin <= P.tol_outer || active == 0) { S.phase = PH_DONE; S.status = 0; break; }
        if (S.s >= P.max_outer) { S.phase = PH_DONE; S.status = 1; break; }
        S.phase = PH_LOB_INIT;
        S.it = 0;
        S.has_p = 0;
        D.act |= A_LOB_SETUP;
        D.usrc = U_DLX;
        break;
    }
    case PH_LOB_INIT: {
        float xax = csum_value(R.s[0]), xx = csum_value(R.s[1]);
        float lam = xx > 0.f ? xax / xx : 0.f;
        S.lam = lam;
        S.has_p = 0;
        S.it = 0;
        D.act |= A_LOB_NORM | A_RESID;
        D.c0 = xx > 0.f ? rsqrtf(xx) : 0.f;
        D.lam = lam;
        S.phase = PH_LOB;
        D.usrc = U_DLW;
        break;
    }
    case PH_LOB: {
        S.it += 1;
        S.lob_iters += 1;
        float ga[6], gb[6];
        for (int t = 0; t < 6; ++t) {
            ga[t] = csum_value(R.s[t]);
            gb[t] = csum_value(R.s[6 + t]);
        }
        bool conv = false;
        float lam_old = S.lam, lam_new = lam_old, c[3] = {1.f, 0.f, 0.f};
        if (!(gb[3] > 0.f)) {
            conv = true;  // zero residual: x is an eigenvector
        } else if (!rayleigh_ritz(ga, gb, S.has_p != 0, lam_new, c)) {
            conv = true;  // breakdown: keep the last Ritz value
            lam_new = lam_old;
        } else if (lam_new > lam_old + 1e-3f * fabsf(lam_old)) {
            conv = true;  // LOBPCG is monotone in exact arithmetic: an increase is noise
            lam_new = lam_old;
        } else {
            conv = (fabsf(lam_new - lam_old) <= P.lob_tol * fmaxf(fabsf(lam_new), 1e-30f) && S.it >= 2) ||
                   S.it >= P.lob_max;
            S.lam = lam_new;
        }
        if (!conv) {
            D.act |= A_LOB_UPDATE | A_RESID;
            D.cx = c[0];
            D.cw = c[1];
            D.cp = c[2];
            D.lam = lam_new;
            S.has_p = 1;
            D.usrc = U_DLW;
            break;
        }
        // Sec. 3.4: alpha = eta * lambda_min.  The paper does not say what to do when
        // lambda_min is not positive or is tiny; below the resolution floor F = c * delta * rho
        // (the smallest curvature change the KKT test of Eq. (cret) can resolve) the step is
        // eta * F * 2^m, m = the floor steps taken in a row just before this one (at most 60)
        float lam = lam_new;
        float F = P.lambda_floor_rel * P.tol_inner * S.rho;
        float alpha;
        if (lam > F) {
            alpha = P.eta * lam;
            S.consec_fb = 0;
        } else {
            alpha = P.eta * ldexpf(F, min(S.consec_fb, 60));
            S.consec_fb += 1;
            S.floor_steps += 1;
        }
        S.lam = lam;
        S.pen_alpha = alpha;
        if (L.stop_after & STOP_LOB) { S.phase = PH_DONE; break; }
        D.act |= A_PENALTY;
        D.alpha = alpha;
        S.phase = PH_INNER;
        S.k = 0;
        D.usrc = U_X;
        break;
    }
    case PH_INNER: {
        S.inner_iters += 1;
        const int k = S.k;
        if (k == 0) {
            S.rho = fmaxf(fmaxf(1.f, 2.f * L.qmax_off), fmaxf(2.f * R.m[1], R.m[2]));
            S.alpha = R.m[3] > 0.f ? 1.f / (2.f * R.m[3]) : 1.f;
        }
        int exit_code = -1;
        if (R.m[0] / S.rho < P.tol_inner) exit_code = 0;
        else if (k >= P.max_inner) exit_code = 1;
        else if (L.method == 1 && k >= 1) {
            // Alg. 1 ends when the projected step left x unchanged (s = x_k - x_{k-1} = 0): in
            // FP32 a step g / (2 h_p) below half an ulp of x stalls the iteration
            if (csum_value(R.s[0]) == 0.f) exit_code = 2;
        } else if (L.method == 0 && k >= 1) {
            float ss = csum_value(R.s[0]), sy = csum_value(R.s[1]), yy = csum_value(R.s[2]);
            if (ss == 0.f) exit_code = 2;
            else {
                float a = (k & 1) ? ss / sy : sy / yy;
                if (!(sy > 0.f) || !isfinite(a)) a = S.alpha;
                a = fminf(fmaxf(a, P.alpha_min), P.alpha_max);
                S.alpha = a;
            }
        }
        if (L.trace_len > 0 && k < L.trace_len && exit_code < 0) {
            D.act |= A_TRACE;
            D.trace_k = k;
        }
        if (L.trace_len > 0 && k < L.trace_len && exit_code >= 0) {
            D.act |= A_TRACE;  // final iterate of the trace
            D.trace_k = k;
        }
        if (exit_code < 0) {
            D.act |= (L.method == 0) ? A_STEP_PABB : A_STEP_PPA;
            D.alpha = S.alpha;
            S.k = k + 1;
            S.inner_steps += 1;
            D.usrc = U_X;
            break;
        }
        S.last_exit = exit_code;
        S.s += 1;
        if (P.hist) atomicAdd((unsigned long long*)&P.hist[min(k / 100, 100)], 1ull);
        if (L.stop_after & STOP_INNER) { S.phase = PH_DONE; break; }
        S.phase = PH_EVAL;
        D.usrc = U_ROUND;
        break;
    }
    default: break;
    }
}

// The reduction of a lane's phase-A partials (all threads of the CTA; the result is in R when
// the call returns).  Thread t merges partials t, t + blockDim.x, ... in order, then the warps
// and the CTA's warps in order: the result depends only on the partials and the CTA size.
// `first`: this thread's first partial (part[threadIdx.x]), when the caller loaded it already.
static __device__ void reduce_partials(const Partial* part, int nblk, int ph, Partial& R,
                                       const Partial* first = nullptr)
{
    Acc a;
    a.zero();
    const int ns = phase_nsum(ph), nm = phase_nmax(ph);
    auto merge = [&](const Partial& p) {
#pragma unroll
        for (int t = 0; t < 12; ++t)
            if (t < ns) a.s[t] = csum_merge(a.s[t], p.s[t]);
#pragma unroll
        for (int t = 0; t < 6; ++t)
            if (t < nm) a.m[t] = fmaxf(a.m[t], p.m[t]);
        a.f += p.f;
    };
    int b0 = threadIdx.x;
    if (first && b0 < nblk) {
        merge(*first);
        b0 += blockDim.x;
    }
    for (int b = b0; b < nblk; b += blockDim.x) merge(part[b]);
    __shared__ float2 sh_s[kBWarps][12];
    __shared__ float sh_m[kBWarps][6];
    __shared__ double sh_f[kBWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    acc_shfl_reduce(a, ph, ph == PH_EVAL);
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < 12; ++t) sh_s[warp][t] = a.s[t];
#pragma unroll
        for (int t = 0; t < 6; ++t) sh_m[warp][t] = a.m[t];
        sh_f[warp] = a.f;
    }
    __syncthreads();
    // the warps' results merged in warp order, one quantity per thread (threads 0-11 the sums,
    // 12-17 the maxima, 18 the FP64 sum): each quantity sees the same operations in the same
    // order as one thread merging them all would
    const int nw = (int)(blockDim.x >> 5);
    const int q = threadIdx.x;
    if (q < 12) {
        float2 v = make_float2(0.f, 0.f);
        for (int w = 0; w < nw; ++w) v = csum_merge(v, sh_s[w][q]);
        R.s[q] = v;
    } else if (q < 18) {
        float v = 0.f;
        for (int w = 0; w < nw; ++w) v = fmaxf(v, sh_m[w][q - 12]);
        R.m[q - 12] = v;
    } else if (q == 18) {
        double v = 0.0;
        if (ph == PH_EVAL)
            for (int w = 0; w < nw; ++w) v += sh_f[w];
        R.f = v;
    }
    __syncthreads();
}

// One 16-byte group q of the projected step: x_prev <- x, x <- P(x - alpha g), u <- x (the
// lane's mode and BF16 input pointers passed in: read from the descriptor after the stores
// here, they would be loaded again, since the compiler cannot rule out that vec aliases it).
__device__ __forceinline__ void pabb_group(int mode, __nv_bfloat16* u_hi, __nv_bfloat16* u_lo, float* vec, int ld,
                                           float al, int q, float4 x, float4 g)
{
    reinterpret_cast<float4*>(vec + (size_t)V_XPREV * ld)[q] = x;
    float4 y;
    y.x = fminf(fmaxf(fmaf(-al, g.x, x.x), 0.f), 1.f);
    y.y = fminf(fmaxf(fmaf(-al, g.y, x.y), 0.f), 1.f);
    y.z = fminf(fmaxf(fmaf(-al, g.z, x.z), 0.f), 1.f);
    y.w = fminf(fmaxf(fmaf(-al, g.w, x.w), 0.f), 1.f);
    reinterpret_cast<float4*>(vec + (size_t)V_X * ld)[q] = y;
    if (mode == MODE_TC) {
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(y.x, y.y), h23 = __floats2bfloat162_rn(y.z, y.w);
        reinterpret_cast<__nv_bfloat162*>(u_hi)[2 * q] = h01;
        reinterpret_cast<__nv_bfloat162*>(u_hi)[2 * q + 1] = h23;
        if (u_lo) {
            const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
            reinterpret_cast<__nv_bfloat162*>(u_lo)[2 * q] = __floats2bfloat162_rn(y.x - f01.x, y.y - f01.y);
            reinterpret_cast<__nv_bfloat162*>(u_lo)[2 * q + 1] = __floats2bfloat162_rn(y.z - f23.x, y.w - f23.y);
        }
    } else {
        reinterpret_cast<float4*>(vec + (size_t)V_U * ld)[q] = y;
    }
}

// The element-wise part of a lane's update for the decision D, over elements [ia, ib) (and,
// for the plain projected step, 16-byte groups [qa, qb) of the padded length).  Every element
// is computed on its own, so a lane's result does not depend on how the range is split.
static __device__ void lane_apply(const LaneDev& L, const Params& P, const Decision& D, int ia, int ib, int qa, int qb,
                                  int tid, int nt)
{
    const int n = L.n, ld = L.ld;
    (void)P;
    float* vec = L.vec;
    const int act = D.act, usrc = D.usrc;
    if (act == A_STEP_PABB && usrc == U_X) {
        // the common tick: x_prev <- x, x <- P(x - alpha g), u <- x over the padded length in
        // 16-byte pieces (padding stays zero: x = g = 0 there)
        const float al = D.alpha;
        const float4* X4 = reinterpret_cast<const float4*>(vec + (size_t)V_X * ld);
        const float4* G4 = reinterpret_cast<const float4*>(vec + (size_t)V_G * ld);
        // two groups per thread per pass, both loaded before either is stored
        for (int q0 = qa + tid; q0 < qb; q0 += 2 * nt) {
            float4 xs[2], gs[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = q0 + h * nt;
                if (q < qb) {
                    xs[h] = X4[q];
                    gs[h] = G4[q];
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = q0 + h * nt;
                if (q >= qb) break;
                pabb_group(L.mode, L.u_hi, L.u_lo, vec, ld, al, q, xs[h], gs[h]);
            }
        }
    }
    for (int i = ia + tid; i < ib && !(act == A_STEP_PABB && usrc == U_X); i += nt) {
        float x = vec[V_X * ld + i];
        if (act & A_TRACE) L.trace_x[(size_t)D.trace_k * n + i] = x;
        if (act & A_COPY_W_X) {
            x = vec[V_W * ld + i];
            vec[V_X * ld + i] = x;
        }
        if (act & A_SAVE_BEST) L.best_x[i] = x > 0.5f ? 1 : 0;
        if (act & A_LOB_SETUP) {
            // Eq. (eq:alpha): z = x - x^2, I_alpha = {z > tau_z}, scaling z^-1/2
            float z = x - x * x;
            bool in = z > P.tau_z;
            float Dz = in ? 1.0f / sqrtf(z) : 0.f;
            float dmp = vec[V_DMP * ld + i];
            vec[V_D * ld + i] = Dz;
            vec[V_T * ld + i] = in ? z / fmaxf(fabsf(dmp), 1e-30f) : 0.f;
            vec[V_LX * ld + i] = in ? start_component(i) : 0.f;
            vec[V_LP * ld + i] = 0.f;
            vec[V_LAP * ld + i] = 0.f;
        }
        if (act & A_LOB_NORM) {
            float lx = vec[V_LX * ld + i] * D.c0;
            vec[V_LX * ld + i] = lx;
            vec[V_LAX * ld + i] = vec[V_W * ld + i] * D.c0;
        }
        if (act & A_LOB_UPDATE) {
            float lx = vec[V_LX * ld + i], lw = vec[V_LW * ld + i], lp = vec[V_LP * ld + i];
            float lax = vec[V_LAX * ld + i], aw = vec[V_W * ld + i], lap = vec[V_LAP * ld + i];
            float np = fmaf(D.cw, lw, D.cp * lp);
            float nap = fmaf(D.cw, aw, D.cp * lap);
            vec[V_LX * ld + i] = fmaf(D.cx, lx, np);
            vec[V_LAX * ld + i] = fmaf(D.cx, lax, nap);
            vec[V_LP * ld + i] = np;
            vec[V_LAP * ld + i] = nap;
        }
        if (act & A_RESID) {
            float r = vec[V_LAX * ld + i] - D.lam * vec[V_LX * ld + i];
            vec[V_LW * ld + i] = vec[V_T * ld + i] * r;
        }
        if (act & A_PENALTY) {
            // Eq. (pp1): p <- p + alpha z with z = x - x^2
            float z = x - x * x;
            float p = fmaf(D.alpha, z, vec[V_P * ld + i]);
            vec[V_P * ld + i] = p;
            vec[V_DMP * ld + i] = L.d[i] - p;
            vec[V_BBAR * ld + i] = L.bprime[i] + p;
        }
        if (act & A_STEP_PABB) {
            // Eq. (x2): x <- P(x - alpha g)
            vec[V_XPREV * ld + i] = x;
            x = fminf(fmaxf(fmaf(-D.alpha, vec[V_G * ld + i], x), 0.f), 1.f);
            vec[V_X * ld + i] = x;
        }
        if (act & A_STEP_PPA) {
            // Eq. (x1): x <- P(x - g / (2 h_p)),  h_p = max(sum_j |Q'_ij| - p_i, eps)
            float hp = fmaxf(L.rabs[i] - vec[V_P * ld + i], D.eps_hp);
            vec[V_XPREV * ld + i] = x;
            x = fminf(fmaxf(x - vec[V_G * ld + i] / (2.f * hp), 0.f), 1.f);
            vec[V_X * ld + i] = x;
        }
        float u;
        switch (usrc) {
        case U_X: u = x; break;
        case U_ROUND: u = x > 0.5f ? 1.f : 0.f; break;
        case U_DLX: u = vec[V_D * ld + i] * vec[V_LX * ld + i]; break;
        case U_DLW: u = vec[V_D * ld + i] * vec[V_LW * ld + i]; break;
        default: u = 0.f; break;
        }
        if (usrc != U_NONE) {
            if (L.mode == MODE_TC) {
                __nv_bfloat16 hi = __float2bfloat16_rn(u);
                L.u_hi[i] = hi;
                if (L.u_lo) L.u_lo[i] = __float2bfloat16_rn(u - __bfloat162float(hi));
            } else {
                vec[V_U * ld + i] = u;
            }
        }
    }
}

// The element-wise part of a LOBPCG iteration that does not end the eigen-solve (act =
// A_LOB_UPDATE | A_RESID, next input u = D w): lane_apply's arithmetic for these flags, with
// the loads of U elements per thread issued before any of their stores.
template <int U>
__device__ __forceinline__ void lob_iteration_apply(const LaneDev& L, const Decision& D, int tid, int nt)
{
    // descriptor fields and decision scalars in registers (stores through vec would make the
    // compiler load them again)
    const int n = L.n, ld = L.ld, mode = L.mode;
    float* vec = L.vec;
    __nv_bfloat16* const u_hi = L.u_hi;
    __nv_bfloat16* const u_lo = L.u_lo;
    const float cw = D.cw, cp = D.cp, cx = D.cx, lam = D.lam;
    for (int i0 = tid; i0 < n; i0 += U * nt) {
        float lx[U], lw[U], lp[U], lax[U], aw[U], lap[U], tt[U], dz[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * nt;
            if (i < n) {
                lx[u] = vec[V_LX * ld + i];
                lw[u] = vec[V_LW * ld + i];
                lp[u] = vec[V_LP * ld + i];
                lax[u] = vec[V_LAX * ld + i];
                aw[u] = vec[V_W * ld + i];
                lap[u] = vec[V_LAP * ld + i];
                tt[u] = vec[V_T * ld + i];
                dz[u] = vec[V_D * ld + i];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * nt;
            if (i >= n) break;
            const float np = fmaf(cw, lw[u], cp * lp[u]);
            const float nap = fmaf(cw, aw[u], cp * lap[u]);
            const float x1 = fmaf(cx, lx[u], np);
            const float ax1 = fmaf(cx, lax[u], nap);
            vec[V_LX * ld + i] = x1;
            vec[V_LAX * ld + i] = ax1;
            vec[V_LP * ld + i] = np;
            vec[V_LAP * ld + i] = nap;
            const float r = ax1 - lam * x1;
            const float w1 = tt[u] * r;
            vec[V_LW * ld + i] = w1;
            const float uu = dz[u] * w1;
            if (mode == MODE_TC) {
                __nv_bfloat16 hi = __float2bfloat16_rn(uu);
                u_hi[i] = hi;
                if (u_lo) u_lo[i] = __float2bfloat16_rn(uu - __bfloat162float(hi));
            } else {
                vec[V_U * ld + i] = uu;
            }
        }
    }
}

// The update of one lane by one CTA of 32..kBThreads threads (a multiple of 32).  Called by
// the stand-alone update kernel and by the CTA that completes a GEMV lane's step.  With at
// most blockDim.x partials every thread merges at most one, so the reduction order (and the
// result) does not depend on the CTA size.  kStaged (the stand-alone kernel, which has the
// registers for it): the thread's first partial and its 16-byte groups of x and g for a
// projected step load together with the lane state, before the phase is known, and LOBPCG
// iterations take lob_iteration_apply; the arithmetic is the same.
template <bool kStaged = false>
static __device__ __noinline__ void lane_update(const LaneDev& L, const Params& P, int32_t* active_count)
{
    __shared__ LaneState S;
    __shared__ Partial R;
    __shared__ Decision D;
    __shared__ int32_t phase0;

    // descriptor fields read once, before any store (the compiler cannot rule out that the
    // stores through vec alias the descriptor and would load them again after each)
    const int mode = L.mode, ld = L.ld;
    if (mode == MODE_GRAD) return;
    float* const vec = L.vec;
    __nv_bfloat16* const u_hi = L.u_hi;
    __nv_bfloat16* const u_lo = L.u_lo;
    LaneState* const st = L.st;
    const int tid = (int)threadIdx.x, nt = (int)blockDim.x, nq = ld >> 2;
    constexpr int kPre = 3;   // groups of x and g per thread loaded ahead
    Partial p0;
    float4 xs[kPre], gs[kPre];
    if (kStaged) {
        if (tid < L.nblk) p0 = L.part[tid];
        const float4* X4 = reinterpret_cast<const float4*>(vec + (size_t)V_X * ld);
        const float4* G4 = reinterpret_cast<const float4*>(vec + (size_t)V_G * ld);
#pragma unroll
        for (int h = 0; h < kPre; ++h) {
            const int q = tid + h * nt;
            if (q < nq) {
                xs[h] = X4[q];
                gs[h] = G4[q];
            }
        }
    }
    if (threadIdx.x == 0) {
        S = *st;
        phase0 = S.phase;
    }
    __syncthreads();
    const int ph = phase0;
    if (ph == PH_DONE) return;

    // ---- reduce the partials of this lane and take its decision
    reduce_partials(L.part, L.nblk, ph, R, kStaged ? &p0 : nullptr);
    if (threadIdx.x == 0) decide(L, S, R, P, D);
    __syncthreads();
    // ---- element-wise update
    if (kStaged && D.act == A_STEP_PABB && D.usrc == U_X) {
        const float al = D.alpha;
#pragma unroll
        for (int h = 0; h < kPre; ++h) {
            const int q = tid + h * nt;
            if (q < nq) pabb_group(mode, u_hi, u_lo, vec, ld, al, q, xs[h], gs[h]);
        }
        if (kPre * nt < nq) lane_apply(L, P, D, 0, L.n, kPre * nt, nq, tid, nt);
    } else if (kStaged && D.act == (A_LOB_UPDATE | A_RESID) && D.usrc == U_DLW) {
        lob_iteration_apply<4>(L, D, tid, nt);
    } else {
        lane_apply(L, P, D, 0, L.n, 0, nq, tid, nt);
    }
    const int act = D.act;
    if (threadIdx.x == 0) {
        if ((act & A_TRACE) && L.trace_alpha) L.trace_alpha[D.trace_k] = D.alpha;
        S.updates += 1;
        if (S.phase == PH_DONE && L.nt_active) atomicSub(L.nt_active, 1);   // phase0 != PH_DONE here
        *st = S;
        if (S.phase != PH_DONE && active_count) atomicAdd(active_count, 1);
    }
}

// Per-warp shared-memory slots of warp_lane_update.
struct WarpUpd {
    LaneState S;
    Partial R;
    Decision D;
};

// The update of one lane by one warp (the tensor-core kernels run it in the epilogue warp
// that finished the lane's last M tile).  Thread t merges partials t, t + 32, ...; with at
// most 32 partials this is the order of lane_update with any CTA size (the cross-warp merge
// there only adds zeros), so both give the same bits.
static __device__ __noinline__ void warp_lane_update(const LaneDev& L, const Params& P, WarpUpd& W,
                                                     int32_t* active_count)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) W.S = *L.st;
    __syncwarp();
    const int ph = W.S.phase;
    if (ph == PH_DONE) return;
    Acc a;
    a.zero();
    const int ns = phase_nsum(ph), nm = phase_nmax(ph);
    for (int b = lane; b < L.nblk; b += 32) {
        const Partial& p = L.part[b];
#pragma unroll
        for (int t = 0; t < 12; ++t)
            if (t < ns) a.s[t] = csum_merge(a.s[t], p.s[t]);
#pragma unroll
        for (int t = 0; t < 6; ++t)
            if (t < nm) a.m[t] = fmaxf(a.m[t], p.m[t]);
        a.f += p.f;
    }
#pragma unroll
    for (int t = 0; t < 12; ++t)
        if (t < ns) a.s[t] = csum_shfl_reduce(a.s[t]);
#pragma unroll
    for (int t = 0; t < 6; ++t)
        if (t < nm) a.m[t] = max_shfl_reduce(a.m[t]);
    if (ph == PH_EVAL) a.f = dsum_shfl_reduce(a.f);
    if (lane == 0) {
        for (int t = 0; t < 12; ++t) W.R.s[t] = t < ns ? a.s[t] : make_float2(0.f, 0.f);
        for (int t = 0; t < 6; ++t) W.R.m[t] = t < nm ? a.m[t] : 0.f;
        W.R.f = ph == PH_EVAL ? a.f : 0.0;
        decide(L, W.S, W.R, P, W.D);
    }
    __syncwarp();
    lane_apply(L, P, W.D, 0, L.n, 0, L.ld >> 2, lane, 32);
    __syncwarp();
    if (lane == 0) {
        if ((W.D.act & A_TRACE) && L.trace_alpha) L.trace_alpha[W.D.trace_k] = W.D.alpha;
        W.S.updates += 1;
        if (W.S.phase == PH_DONE && L.nt_active) atomicSub(L.nt_active, 1);
        *L.st = W.S;
        if (W.S.phase != PH_DONE && active_count) atomicAdd(active_count, 1);
    }
    __syncwarp();
}

}  // namespace ubqp
