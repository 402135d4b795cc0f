// FP32 lanes (an instance solved from one start: the plain FP32 path), each as a persistent
// run of many steps of Alg. 3 with Alg. 2 (or Alg. 1), in one cooperative launch.
//
// The CTAs form groups; group g owns CTAs gcta[g] .. gcta[g+1]-1 and runs its lanes one after
// another (one group and one lane for a single instance).  A step of a lane is the
// matrix-vector product of the lane's phase over the group's CTAs, then its update.  CTA c of
// the group owns row blocks c, c + C, ... (C CTAs, rows_per_item rows per block) and a
// contiguous slice of the elements.  Per step:
//   1. every CTA loads u, computes its blocks' rows and row epilogues with the same functions
//      as the other schedulers (gemv_rows.cuh) and writes one partial record per block;
//   2. group barrier;
//   3. every CTA reduces all partial records in the same order (reduce_partials) and takes the
//      same decision (decide) on its own copy of the lane state, so all copies stay equal;
//      then it applies the element-wise update (lane_apply) to its slice;
//   4. group barrier (u complete).
// Alg. 2 steps (PABB) take one barrier: every CTA holds the whole x_k and x_{k-1} in shared
// memory, and after the barrier computes the whole x_{k+1} = P(x_k - alpha g_k) itself from g_k
// (every CTA's rows are in global memory by then), instead of updating a slice and exchanging
// it.  g alternates between two global buffers by the parity of k (V_G, V_W), and so do the
// blocks' partial records (the lane holds two sets), so a CTA that has passed the step's barrier
// and computes step k+1 never overwrites g_k or a record of step k that another CTA of the
// group may still be reading.  On the sliced storage with one slice per block, a CTA computes
// its slices one after another, each with sixteen entries per thread in flight.  When the subproblem ends,
// or the launch's budget does, the CTAs write x_k, x_{k-1} and u back.  The arithmetic is that
// of the lock-step scheduler with the same rows per item, so both give the same bits.  Every
// group barrier wait is bounded: when it runs out the CTA sets the error flag and leaves, and
// the others leave at their own next wait.  A group of one CTA needs no barrier.
//
// Lane vectors and partial records written by one CTA are read by others within the launch,
// so this file is compiled with plain loads cached in L2 only (-dlcm=cg); Q keeps its
// non-coherent streaming loads.
#include "gemv_rows.cuh"

namespace ubqp {

__device__ __forceinline__ uint64_t solo_clock()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Group barrier on a monotonic 64-bit arrival counter: barrier number gen + 1 of the group is
// complete when the counter reaches nc * (gen + 1).  A CTA adds its arrival without waiting for
// the result and polls the counter (bounded); nobody resets anything, so a barrier costs one
// round trip after the last arrival.
__device__ __forceinline__ bool solo_grid_sync(const SoloArgs& A, unsigned long long* bar, int nc,
                                               unsigned long long& gen, int* s_ok)
{
    __syncthreads();
    if (nc == 1) return *s_ok != 0;
    if (threadIdx.x == 0) {
        const unsigned long long target = (gen + 1ull) * (unsigned long long)nc;
        __threadfence();
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
        const uint64_t t0 = solo_clock();
        while (ld_acquire_u64(bar) < target) {
            if (solo_clock() - t0 > A.wait_ns) {
                atomicExch(A.err, 1);
                *s_ok = 0;
                break;
            }
        }
        gen += 1ull;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Alg. 2 row epilogue of the single-barrier step for row i: x_k, x_{k-1}, d - p, d + b' and
// g_{k-1} of the row given, g_k written to gnew[i] and returned; the arithmetic of row_epilogue
// (PH_INNER)
__device__ __forceinline__ float solo_inner_row(const LaneDev& L, int k, int i, float v, float x, float xp, float dmp,
                                                float tsum, float gold, float* gnew, Acc& a)
{
    const float g = fmaf(dmp, 2.f * x - 1.f, fmaf(2.f, v, tsum));
    if (k >= 1) {
        const float sd = x - xp;
        const float y = g - gold;
        csum_add(a.s[0], sd * sd);
        csum_add(a.s[1], sd * y);
        csum_add(a.s[2], y * y);
    } else {
        a.m[1] = fmaxf(a.m[1], fabsf(dmp));
        a.m[2] = fmaxf(a.m[2], fabsf(L.vec[V_BBAR * L.ld + i]));
        a.m[3] = fmaxf(a.m[3], L.oabs[i] + fabsf(dmp));
    }
    gnew[i] = g;
    const float viol = (x > 0.f && x < 1.f) ? fabsf(g) : (x <= 0.f ? fmaxf(-g, 0.f) : fmaxf(g, 0.f));
    a.m[0] = fmaxf(a.m[0], viol);
    return g;
}

__device__ __forceinline__ unsigned long long solo_item_bytes(const LaneDev& L, int blk, int row0, int rows)
{
    if (L.spv)
        return 6ull * (unsigned long long)(L.spo[(row0 + rows + 31) >> 5] - L.spo[row0 >> 5]) +
               (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
    return (unsigned long long)rows * L.n * 4ull + (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
}

// the row epilogue of one block and its partial record, by the whole CTA
__device__ __forceinline__ void solo_inner_finish(const LaneDev& L, int k, int blk, int row0, int rows,
                                                  const double* sv, const Params& P, const float* sx,
                                                  const float* sxp, const float* gold, float* gnew,
                                                  const float* dmpv, const float* tsumv, Partial* out)
{
    Acc a;
    a.zero();
    if ((int)threadIdx.x < rows) {
        const int i = row0 + threadIdx.x;
        solo_inner_row(L, k, i, (float)sv[threadIdx.x], sx[i], sxp[i], dmpv[i], tsumv[i], k >= 1 ? gold[i] : 0.f, gnew, a);
    }
    block_reduce_write<kWarps>(a, PH_INNER, out, false);
    if (P.bytes && threadIdx.x == 0) atomicAdd(P.bytes, solo_item_bytes(L, blk, row0, rows));
}

// The same epilogue and record for a block of at most 32 rows, by one warp (lane r: row r).
// block_reduce_write over the CTA would merge this warp's sums with seven warps' zero sums in
// warp order; the merges below are those, so the record has the same bits.
__device__ __forceinline__ void solo_inner_finish_warp(const LaneDev& L, int k, int blk, int row0, int rows,
                                                       const double* sv, const Params& P, const float* sx,
                                                       const float* sxp, float* gnew, float dmp, float tsum,
                                                       float gold, Partial* out, int lane)
{
    Acc a;
    a.zero();
    if (lane < rows) {
        const int i = row0 + lane;
        solo_inner_row(L, k, i, (float)sv[lane], sx[i], sxp[i], dmp, tsum, gold, gnew, a);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) a.s[t] = csum_shfl_reduce(a.s[t]);
#pragma unroll
    for (int t = 0; t < 4; ++t) a.m[t] = max_shfl_reduce(a.m[t]);
    if (lane == 0) {
        Partial R;
        const float2 z2 = make_float2(0.f, 0.f);
        for (int t = 0; t < 12; ++t) R.s[t] = z2;
        for (int t = 0; t < 6; ++t) R.m[t] = 0.f;
        R.f = 0.0;
        const int ns = phase_nsum(PH_INNER), nm = phase_nmax(PH_INNER);
        for (int t = 0; t < ns; ++t) R.s[t] = csum_merge(R.s[t], a.s[t]);
        for (int t = 0; t < nm; ++t) R.m[t] = fmaxf(R.m[t], a.m[t]);
        R.f += 0.0;
        for (int w = 1; w < kWarps; ++w) {
            for (int t = 0; t < ns; ++t) R.s[t] = csum_merge(R.s[t], z2);
            for (int t = 0; t < nm; ++t) R.m[t] = fmaxf(R.m[t], 0.f);
            R.f += 0.0;
        }
        *out = R;
        if (P.bytes) atomicAdd(P.bytes, solo_item_bytes(L, blk, row0, rows));
    }
}

// Products of one 32-row slice (sliced storage) for sv[r]: the shares, operations and merge of
// item_rows_sell with eight warps per slice, the loads sixteen entries of the share at a time
// (a CTA with a single slice waits for fewer load rounds)
__device__ __forceinline__ void solo_rows_one(const LaneDev& L, int sl, int rows, const float* su, double* sv,
                                              float2* s_share1, int lane, int warp)
{
    const int64_t base = L.spo[sl];
    const int width = (int)((L.spo[sl + 1] - base) >> 5);
    const int k0 = width * warp / kWarps, k1 = width * (warp + 1) / kWarps;
    const float* V = L.spv + base + lane + 32 * (int64_t)k0;
    const uint16_t* C = L.spc + base + lane + 32 * (int64_t)k0;
    const int ng = ((k1 - k0) >> 3) * 2;   // groups of four summed as FMA groups
    float2 acc = make_float2(0.f, 0.f);
    int j = 0;
    for (; j + 4 <= ng; j += 4) {
        float q[16];
        int c[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            q[e] = __ldg(V + 32 * (4 * j + e));
            c[e] = __ldg(C + 32 * (4 * j + e));
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float t = __fmul_rn(q[4 * h], su[c[4 * h]]);
            t = fmaf(q[4 * h + 1], su[c[4 * h + 1]], t);
            t = fmaf(q[4 * h + 2], su[c[4 * h + 2]], t);
            t = fmaf(q[4 * h + 3], su[c[4 * h + 3]], t);
            csum_add(acc, t);
        }
    }
    for (; j < ng; ++j) {
        float q[4];
        int c[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            q[e] = __ldg(V + 32 * (4 * j + e));
            c[e] = __ldg(C + 32 * (4 * j + e));
        }
        float t = __fmul_rn(q[0], su[c[0]]);
        t = fmaf(q[1], su[c[1]], t);
        t = fmaf(q[2], su[c[2]], t);
        t = fmaf(q[3], su[c[3]], t);
        csum_add(acc, t);
    }
    for (int k = 4 * ng; k < k1 - k0; ++k) csum_add(acc, __fmul_rn(__ldg(V + 32 * k), su[__ldg(C + 32 * k)]));
    s_share1[lane * kWarps + warp] = acc;
    __syncthreads();
    if ((int)threadIdx.x < rows) {
        const float2* sh = s_share1 + threadIdx.x * kWarps;
        float2 a = sh[0];
        for (int w = 1; w < kWarps; ++w) a = csum_merge(a, sh[w]);
        sv[threadIdx.x] = (double)(a.x + a.y);
    }
}

// x_{k+1} = P(x_k - alpha g_k) over the whole padded vector (ld a multiple of 4), g_k from global
// memory: 16-byte pieces, the loads of up to four pieces per thread issued before any use, so
// the update costs one L2 round trip for ld <= 4096
__device__ __forceinline__ void solo_project(const float* __restrict__ g, const float* x, float* y, int ld, float al)
{
    const float4* g4 = reinterpret_cast<const float4*>(g);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* y4 = reinterpret_cast<float4*>(y);
    const int nq = ld >> 2;
    for (int q0 = threadIdx.x; q0 < nq; q0 += 4 * kThreads) {
        float4 gv[4];
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if (q0 + h * kThreads < nq) gv[h] = g4[q0 + h * kThreads];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int q = q0 + h * kThreads;
            if (q < nq) {
                const float4 xv = x4[q];
                float4 r;
                r.x = fminf(fmaxf(fmaf(-al, gv[h].x, xv.x), 0.f), 1.f);
                r.y = fminf(fmaxf(fmaf(-al, gv[h].y, xv.y), 0.f), 1.f);
                r.z = fminf(fmaxf(fmaf(-al, gv[h].z, xv.z), 0.f), 1.f);
                r.w = fminf(fmaxf(fmaf(-al, gv[h].w, xv.w), 0.f), 1.f);
                y4[q] = r;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) solo_lane_kernel(SoloArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sv[kThreads];
    __shared__ LaneState S;
    __shared__ Partial R;
    __shared__ Decision D;
    __shared__ int s_ok, s_g;
    __shared__ unsigned long long s_gen0;
    __shared__ float2 s_share[kSoloMaxSl][kThreads];
    __shared__ Partial s_part;
    // the descriptor never changes: one copy in shared memory (this file's plain loads go to
    // L2, so every field read from global memory would be an L2 round trip)
    __shared__ __align__(16) LaneDev sL;
    static_assert(sizeof(LaneDev) % 8 == 0, "descriptor copied in 8-byte pieces");

    // ---- this CTA's group, its rank in the group and the group's barrier
    if (threadIdx.x == 0) {
        int g = 0;
        if (A.gcta) {
            int lo = 0, hi = A.ngroups - 1;   // the last group whose first CTA is <= blockIdx.x
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.gcta[mid] <= (int)blockIdx.x) lo = mid;
                else hi = mid - 1;
            }
            g = lo;
        }
        s_g = g;
        s_ok = 1;
    }
    __syncthreads();
    const int g = s_g;
    const int c0 = A.gcta ? A.gcta[g] : 0;
    const int nc = A.gcta ? A.gcta[g + 1] - c0 : (int)gridDim.x;
    const int rank = (int)blockIdx.x - c0;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(A.bar + (size_t)g * kSoloBarStride);
    // barriers the group completed in earlier launches (a CTA that is already waiting at this
    // launch's first barrier has added less than nc)
    if (threadIdx.x == 0) s_gen0 = ld_acquire_u64(bar) / (unsigned long long)nc;
    __syncthreads();
    unsigned long long gen = s_gen0;
    // the parameters in shared memory (read rarely; as a register copy they crowd the products'
    // loop); the subproblem histogram is counted once per lane, by the group's first CTA
    __shared__ Params sP;
    if (threadIdx.x == 0) {
        sP = A.P;
        if (rank != 0) sP.hist = nullptr;
    }
    __syncthreads();
    const Params& P = sP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int li0 = A.glanes ? A.gfirst[g] : 0, li1 = A.glanes ? A.gfirst[g + 1] : 1;
    int steps_left = A.budget;

    for (int li = li0; li < li1 && steps_left > 0; ++li) {
        const int lane_id = A.glanes ? A.glanes[li] : 0;
        __syncthreads();   // shared state of the previous lane no longer in use
        if (threadIdx.x < (int)(sizeof(LaneDev) / 8))
            reinterpret_cast<int2*>(&sL)[threadIdx.x] =
                __ldg(reinterpret_cast<const int2*>(A.lane + lane_id) + threadIdx.x);
        __syncthreads();
        const LaneDev& L = sL;
        if (threadIdx.x == 0) S = *L.st;
        __syncthreads();
        if (S.phase == PH_DONE) continue;
        const int nblk = L.nblk;
        const int ng = L.ld >> 2;
        const int qa = (int)((int64_t)ng * rank / nc), qb = (int)((int64_t)ng * (rank + 1) / nc);
        const int ia = min(4 * qa, L.n), ib = min(4 * qb, L.n);

        // single-barrier Alg. 2 state: su = x_k and sxp = x_{k-1} (whole vectors) while fast is set
        float* su = reinterpret_cast<float*>(smem_raw);
        float* sxp = su + L.ld;
        bool fast = false;
        const bool pabb = L.method == 0;
        float* gbuf[2] = {L.vec + (size_t)V_G * L.ld, L.vec + (size_t)V_W * L.ld};
        // One CTA for a lane of one block: during Alg. 2 the g buffers, d - p and d + b' live in
        // shared memory and the step's partial record stays there too, so a step reads only the
        // rows of Q from global memory.  The g buffers are loaded at the start and stored at the
        // end of a launch that stops inside a subproblem.
        const bool one = nc == 1 && nblk == 1 && A.fast && A.one_ok;
        float* sdmp = sxp + L.ld;
        float* stsum = sdmp + L.ld;
        const float* dmpv = L.vec + (size_t)V_DMP * L.ld;
        const float* tsumv = L.tsum;
        if (one) {
            float* sg = stsum + L.ld;
            for (int c = threadIdx.x; c < L.ld; c += kThreads) {
                sg[c] = gbuf[0][c];
                sg[L.ld + c] = gbuf[1][c];
            }
            gbuf[0] = sg;
            gbuf[1] = sg + L.ld;
            dmpv = sdmp;
            tsumv = stsum;
            __syncthreads();
        }
        // this CTA's blocks (sliced storage, 32 rows per item: all of them before one barrier)
        const bool multi = L.spv && A.rows_per_item == 32 && (nblk + nc - 1) / nc <= kSoloMaxSl;
        int my_sl[kSoloMaxSl];
        int my_n = 0;
#pragma unroll
        for (int b = 0; b < kSoloMaxSl; ++b) {
            const int blk = rank + b * nc;
            my_sl[b] = blk;
            if (blk < nblk) my_n = b + 1;
        }

        for (; steps_left > 0; --steps_left) {
            const int ph = S.phase;
            if (ph == PH_DONE) break;
            const int k = S.k;
            const bool fast_step = A.fast && pabb && ph == PH_INNER;
            if (!fast) {
                item_load_u(L, su);
                if (fast_step && k >= 1)
                    for (int c = threadIdx.x; c < L.ld; c += kThreads) sxp[c] = L.vec[(size_t)V_XPREV * L.ld + c];
                if (fast_step && one)   // d - p and d + b' are fixed for the subproblem
                    for (int c = threadIdx.x; c < L.ld; c += kThreads) {
                        sdmp[c] = L.vec[(size_t)V_DMP * L.ld + c];
                        stsum[c] = L.tsum[c];
                    }
                __syncthreads();
            }
            // ---- phase A: this CTA's row block(s)
            if (fast_step && multi) {
                if (my_n > 0) {
                    // the epilogue's per-row operands of warp w's block (d - p, d + b', g_{k-1}),
                    // loaded before the products so that their round trip overlaps them
                    float e_dmp = 0.f, e_ts = 0.f, e_g = 0.f;
                    if (warp < my_n) {
                        const int i = min(my_sl[warp] * 32 + lane, L.n - 1);
                        e_dmp = dmpv[i];
                        e_ts = tsumv[i];
                        if (k >= 1) e_g = gbuf[(k + 1) & 1][i];
                    }
                    // the CTA's slices one after another, each into its own share buffer (measured
                    // faster than interleaving the slices' loads, which cost registers)
                    for (int b = 0; b < my_n; ++b)
                        solo_rows_one(L, my_sl[b], min(32, L.n - my_sl[b] * 32), su, sv + 32 * b, s_share[b], lane, warp);
                    __syncthreads();
                    if (warp < my_n) {
                        const int blk = my_sl[warp], row0 = blk * 32;
                        solo_inner_finish_warp(L, k, blk, row0, min(32, L.n - row0), sv + 32 * warp, P, su, sxp,
                                               gbuf[k & 1], e_dmp, e_ts, e_g,
                                               one ? &s_part : L.part + (size_t)(k & 1) * nblk + blk, lane);
                    }
                }
            } else {
                for (int blk = rank; blk < nblk; blk += nc) {
                    const int row0 = blk * A.rows_per_item;
                    const int rows = min(A.rows_per_item, L.n - row0);
                    item_rows_solver(L, ph, row0, rows, su, sv, lane, warp);
                    __syncthreads();
                    if (fast_step)
                        solo_inner_finish(L, k, blk, row0, rows, sv, P, su, sxp, gbuf[(k + 1) & 1], gbuf[k & 1], dmpv,
                                          tsumv, one ? &s_part : L.part + (size_t)(k & 1) * nblk + blk);
                    else item_finish(L, ph, k, blk, row0, rows, sv, P);
                    __syncthreads();
                }
            }
            if (!solo_grid_sync(A, bar, nc, gen, &s_ok)) break;
            // ---- the update: the same reduction and decision in every CTA (one CTA in Alg. 2: its
            // single partial record, which the reduction would return unchanged)
            if (fast_step && one) {
                if (threadIdx.x == 0) R = s_part;
                __syncthreads();
            } else {
                reduce_partials(fast_step ? L.part + (size_t)(k & 1) * nblk : L.part, nblk, ph, R);
            }
            // (decide and lane_apply stay inlined: built out of line in this file, with its plain
            // loads cached in L2 only, their reads of the shared-memory state through generic
            // references returned wrong values on the GPU)
            if (threadIdx.x == 0) decide(L, S, R, P, D);
            __syncthreads();
            if (fast_step && (D.act & ~A_TRACE) == A_STEP_PABB && D.usrc == U_X) {
                // x_{k+1} = P(x_k - alpha g_k) for every element, into the x_{k-1} buffer; the trace
                // (x_k) is written for this CTA's slice
                const float al = D.alpha;
                if (D.act & A_TRACE)
                    for (int i = ia + (int)threadIdx.x; i < ib; i += kThreads)
                        L.trace_x[(size_t)D.trace_k * L.n + i] = su[i];
                __syncthreads();
                solo_project(gbuf[k & 1], su, sxp, L.ld, al);
                __syncthreads();
                float* t = su;
                su = sxp;
                sxp = t;
                fast = true;
                if (threadIdx.x == 0) {
                    S.updates += 1;
                    if (rank == 0 && (D.act & A_TRACE) && L.trace_alpha) L.trace_alpha[D.trace_k] = D.alpha;
                }
                __syncthreads();
                continue;
            }
            if (fast_step) {
                // the subproblem ends (or the step is not a plain projected step): this CTA's slice
                // of x_k, x_{k-1} and g_k back to the lane's vectors, then the general update
                const float* gk = gbuf[k & 1];
                for (int i = ia + (int)threadIdx.x; i < ib; i += kThreads) {
                    L.vec[(size_t)V_X * L.ld + i] = su[i];
                    L.vec[(size_t)V_XPREV * L.ld + i] = sxp[i];
                    L.vec[(size_t)V_G * L.ld + i] = gk[i];
                }
                __syncthreads();
                fast = false;
                // the buffers may have traded places: x_k goes back to the start of shared memory
                su = reinterpret_cast<float*>(smem_raw);
                sxp = su + L.ld;
            }
            lane_apply(L, P, D, ia, ib, qa, qb, (int)threadIdx.x, (int)blockDim.x);
            if (threadIdx.x == 0) {
                S.updates += 1;
                if (rank == 0 && (D.act & A_TRACE) && L.trace_alpha) L.trace_alpha[D.trace_k] = D.alpha;
            }
            if (!solo_grid_sync(A, bar, nc, gen, &s_ok)) break;
        }
        if (fast) {
            // the launch ends inside a subproblem: x_k (also the next u) and x_{k-1} back to the lane
            for (int i = ia + (int)threadIdx.x; i < ib; i += kThreads) {
                L.vec[(size_t)V_X * L.ld + i] = su[i];
                L.vec[(size_t)V_U * L.ld + i] = su[i];
                L.vec[(size_t)V_XPREV * L.ld + i] = sxp[i];
            }
            if (one)   // and the g buffers
                for (int c = threadIdx.x; c < L.ld; c += kThreads) {
                    L.vec[(size_t)V_G * L.ld + c] = gbuf[0][c];
                    L.vec[(size_t)V_W * L.ld + c] = gbuf[1][c];
                }
            // padding of u beyond n stays zero (x is zero there)
            for (int i = L.n + (int)threadIdx.x + rank * kThreads; i < L.ld; i += kThreads * nc)
                L.vec[(size_t)V_U * L.ld + i] = 0.f;
        }
        __syncthreads();
        if (rank == 0 && threadIdx.x == 0) *L.st = S;
        if (!s_ok) break;
    }
    // ---- the group's lanes still unfinished (rank 0 wrote the state of every lane it ran)
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0) {
        int left = 0;
        for (int li = li0; li < li1; ++li) {
            const int lane_id = A.glanes ? A.glanes[li] : 0;
            left += A.lane[lane_id].st->phase != PH_DONE ? 1 : 0;
        }
        if (left) atomicAdd(A.active_after, left);
    }
}

// CTAs and rows per block of a lane of n rows: one CTA up to 256 rows, else as many CTAs as
// SMs (at most one per 8 rows), rows split evenly in multiples of 8 (or the caller's count)
void solo_shape(int n, int rows_per_item, int sms, int* grid, int* rb, int* nblk)
{
    int r;
    if (rows_per_item > 0) r = rows_per_item;
    else if (n <= kThreads) r = n;
    else {
        const int g = std::min(sms, (n + 7) / 8);
        r = ((n + g - 1) / g + 7) / 8 * 8;
    }
    r = std::max(1, std::min(r, kThreads));
    *rb = r;
    *nblk = (n + r - 1) / r;
    *grid = std::min(*nblk, sms);
}

size_t solo_smem(int ld, bool one) { return (one ? 6 : 2) * (size_t)ld * sizeof(float); }

cudaError_t prepare_solo(int ld, bool one)
{
    const size_t smem = solo_smem(ld, one);
    // always opted in: the static shared memory counts against the 48 KB default as well
    return cudaFuncSetAttribute(solo_lane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// CTAs of the kernel resident on one SM with the dynamic shared memory of lanes of ld
int solo_ctas_per_sm(int ld, bool one)
{
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solo_lane_kernel, kThreads, solo_smem(ld, one)) !=
        cudaSuccess) {
        cudaGetLastError();
        per = 0;
    }
    return per;
}

// every CTA must be resident: a cooperative launch fails instead of starting a grid that
// could not be
cudaError_t launch_solo(const SoloArgs& a, int ld, cudaStream_t s)
{
    SoloArgs args = a;
    void* params[] = {&args};
    return cudaLaunchCooperativeKernel((const void*)solo_lane_kernel, dim3((unsigned)a.grid), dim3(kThreads), params,
                                       solo_smem(ld, a.one_ok != 0), s);
}

}  // namespace ubqp
