// One FP32 lane (a single instance solved from a single start: the plain FP32 path) as one
// persistent launch that runs many steps of Alg. 3 with Alg. 2 (or Alg. 1).
//
// A step is the matrix-vector product of the lane's phase over all CTAs, then its update.
// CTA c owns row block c of the lane (rows_per_item rows, as many blocks as CTAs) and a
// contiguous slice of the elements.  Per step:
//   1. every CTA loads u, computes its block's rows and row epilogue with the same functions as
//      the other schedulers (gemv_rows.cuh) and writes the block's partial record;
//   2. grid barrier;
//   3. every CTA reduces all partial records in the same order (reduce_partials) and takes the
//      same decision (decide) on its own copy of the lane state, so all copies stay equal;
//      then it applies the element-wise update (lane_apply) to its slice;
//   4. grid barrier (u complete).
// Alg. 2 steps (PABB) take one barrier: every CTA holds the whole x_k and x_{k-1} in shared
// memory, and after the barrier computes the whole x_{k+1} = P(x_k - alpha g_k) itself from g_k
// (every CTA's rows are in global memory by then), instead of updating a slice and exchanging
// it.  g alternates between two global buffers by the parity of k (V_G, V_W), so a CTA that
// writes g_{k+1} never overwrites the g_k another CTA may still be reading.  When the
// subproblem ends, or the launch's budget does, the CTAs write x_k, x_{k-1} and u back.
// The arithmetic is that of the lock-step scheduler with the same rows per item, so both give
// the same bits.  The launch is cooperative (every CTA resident), and each barrier wait is
// bounded: when it runs out the CTA sets the error flag and leaves, and the others leave at
// their own next wait.  With one CTA (n <= 256) the barriers are the CTA's own.
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

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// sense by generation: bar[0] counts arrivals, bar[1] is the generation released so far
__device__ __forceinline__ bool solo_grid_sync(const SoloArgs& A, unsigned& gen, int* s_ok)
{
    __syncthreads();
    if (gridDim.x == 1) return *s_ok != 0;
    if (threadIdx.x == 0) {
        const unsigned target = gen + 1u;
        __threadfence();
        if (atomicAdd(&A.bar[0], 1u) == gridDim.x - 1u) {
            A.bar[0] = 0u;
            __threadfence();
            atomicExch(&A.bar[1], target);
        } else {
            const uint64_t t0 = solo_clock();
            while (ld_acquire_u32(&A.bar[1]) != target) {
                if (solo_clock() - t0 > A.wait_ns) {
                    atomicExch(A.err, 1);
                    *s_ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        gen = target;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Alg. 2 row epilogue of the single-barrier step: the arithmetic of row_epilogue (PH_INNER)
// with x_k and x_{k-1} from shared memory, g_{k-1} from gold and g_k written to gnew
__device__ __forceinline__ void solo_inner_finish(const LaneDev& L, int k, int blk, int row0, int rows,
                                                  const double* sv, const Params& P, const float* sx,
                                                  const float* sxp, const float* gold, float* gnew,
                                                  const float* dmpv, const float* tsumv, Partial* out)
{
    Acc a;
    a.zero();
    const int ld = L.ld;
    if ((int)threadIdx.x < rows) {
        const int i = row0 + threadIdx.x;
        const float v = (float)sv[threadIdx.x];
        const float x = sx[i];
        const float dmp = dmpv[i];
        const float g = fmaf(dmp, 2.f * x - 1.f, fmaf(2.f, v, tsumv[i]));
        if (k >= 1) {
            const float sd = x - sxp[i];
            const float y = g - gold[i];
            csum_add(a.s[0], sd * sd);
            csum_add(a.s[1], sd * y);
            csum_add(a.s[2], y * y);
        } else {
            a.m[1] = fmaxf(a.m[1], fabsf(dmp));
            a.m[2] = fmaxf(a.m[2], fabsf(L.vec[V_BBAR * ld + i]));
            a.m[3] = fmaxf(a.m[3], L.oabs[i] + fabsf(dmp));
        }
        gnew[i] = g;
        const float viol = (x > 0.f && x < 1.f) ? fabsf(g) : (x <= 0.f ? fmaxf(-g, 0.f) : fmaxf(g, 0.f));
        a.m[0] = fmaxf(a.m[0], viol);
    }
    block_reduce_write<kWarps>(a, PH_INNER, out, false);
    if (P.bytes && threadIdx.x == 0) {
        unsigned long long by = (unsigned long long)rows * L.n * 4ull + (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
        if (L.spv)
            by = 6ull * (unsigned long long)(L.spo[(row0 + rows + 31) >> 5] - L.spo[row0 >> 5]) +
                 (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
        atomicAdd(P.bytes, by);
    }
}

__global__ void __launch_bounds__(kThreads, 1) solo_lane_kernel(SoloArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* su = reinterpret_cast<float*>(smem_raw);
    __shared__ double sv[kThreads];
    __shared__ LaneState S;
    __shared__ Partial R;
    __shared__ Decision D;
    __shared__ int s_ok;
    __shared__ unsigned s_gen0;
    // the descriptor never changes: one copy in shared memory (this file's plain loads go to
    // L2, so every field read from global memory would be an L2 round trip)
    __shared__ __align__(16) LaneDev sL;
    static_assert(sizeof(LaneDev) % 8 == 0, "descriptor copied in 8-byte pieces");
    if (threadIdx.x < (int)(sizeof(LaneDev) / 8))
        reinterpret_cast<int2*>(&sL)[threadIdx.x] = __ldg(reinterpret_cast<const int2*>(A.lane) + threadIdx.x);
    __syncthreads();
    const LaneDev& L = sL;
    if (threadIdx.x == 0) {
        S = *L.st;
        s_ok = 1;
        s_gen0 = ld_acquire_u32(&A.bar[1]);
    }
    __syncthreads();
    unsigned gen = s_gen0;
    Params P = A.P;
    if (blockIdx.x != 0) P.hist = nullptr;   // the subproblem histogram is counted once
    const int ng = L.ld >> 2;
    const int qa = (int)((int64_t)ng * blockIdx.x / gridDim.x), qb = (int)((int64_t)ng * (blockIdx.x + 1) / gridDim.x);
    const int ia = min(4 * qa, L.n), ib = min(4 * qb, L.n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // single-barrier Alg. 2 state: su = x_k and sxp = x_{k-1} (whole vectors) while fast is set
    float* sxp = su + L.ld;
    bool fast = false;
    const bool pabb = L.method == 0;
    float* gbuf[2] = {L.vec + (size_t)V_G * L.ld, L.vec + (size_t)V_W * L.ld};
    // One CTA (n <= 256): during Alg. 2 the g buffers, d - p and d + b' live in shared memory
    // and the step's partial record stays there too, so a step reads only the rows of Q from
    // global memory.  The g buffers are loaded at the start and stored at the end of a launch
    // that stops inside a subproblem.
    const bool one = gridDim.x == 1 && A.fast != 0;
    __shared__ Partial s_part;
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

    for (int step = 0; step < A.budget; ++step) {
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
        for (int blk = blockIdx.x; blk < A.nblk; blk += gridDim.x) {
            const int row0 = blk * A.rows_per_item;
            const int rows = min(A.rows_per_item, L.n - row0);
            item_rows_solver(L, ph, row0, rows, su, sv, lane, warp);
            __syncthreads();
            if (fast_step)
                solo_inner_finish(L, k, blk, row0, rows, sv, P, su, sxp, gbuf[(k + 1) & 1], gbuf[k & 1], dmpv, tsumv,
                                  one ? &s_part : L.part + blk);
            else item_finish(L, ph, k, blk, row0, rows, sv, P);
            __syncthreads();
        }
        if (!solo_grid_sync(A, gen, &s_ok)) break;
        // ---- the update: the same reduction and decision in every CTA (one CTA in Alg. 2: its
        // single partial record, which the reduction would return unchanged)
        if (fast_step && one) {
            if (threadIdx.x == 0) R = s_part;
            __syncthreads();
        } else {
            reduce_partials(L.part, A.nblk, ph, R);
        }
        if (threadIdx.x == 0) decide(L, S, R, P, D);
        __syncthreads();
        if (fast_step && (D.act & ~A_TRACE) == A_STEP_PABB && D.usrc == U_X) {
            // x_{k+1} = P(x_k - alpha g_k) for every element, into the x_{k-1} buffer; the trace
            // (x_k) is written for this CTA's slice
            const float al = D.alpha;
            const float* g = gbuf[k & 1];
            if (D.act & A_TRACE)
                for (int i = ia + (int)threadIdx.x; i < ib; i += kThreads) L.trace_x[(size_t)D.trace_k * L.n + i] = su[i];
            __syncthreads();
            for (int i = threadIdx.x; i < L.ld; i += kThreads) sxp[i] = fminf(fmaxf(fmaf(-al, g[i], su[i]), 0.f), 1.f);
            __syncthreads();
            float* t = su;
            su = sxp;
            sxp = t;
            fast = true;
            if (threadIdx.x == 0) {
                S.updates += 1;
                if (blockIdx.x == 0 && (D.act & A_TRACE) && L.trace_alpha) L.trace_alpha[D.trace_k] = D.alpha;
            }
            __syncthreads();
            continue;
        }
        if (fast_step) {
            // the subproblem ends (or the step is not a plain projected step): this CTA's slice of
            // x_k, x_{k-1} and g_k back to the lane's vectors, then the general update
            const float* g = gbuf[k & 1];
            for (int i = ia + (int)threadIdx.x; i < ib; i += kThreads) {
                L.vec[(size_t)V_X * L.ld + i] = su[i];
                L.vec[(size_t)V_XPREV * L.ld + i] = sxp[i];
                L.vec[(size_t)V_G * L.ld + i] = g[i];
            }
            __syncthreads();
            fast = false;
        }
        lane_apply(L, P, D, ia, ib, qa, qb, (int)threadIdx.x, (int)blockDim.x);
        if (threadIdx.x == 0) {
            S.updates += 1;
            if (blockIdx.x == 0 && (D.act & A_TRACE) && L.trace_alpha) L.trace_alpha[D.trace_k] = D.alpha;
        }
        if (!solo_grid_sync(A, gen, &s_ok)) break;
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
        for (int i = L.n + (int)threadIdx.x + (int)blockIdx.x * kThreads; i < L.ld; i += kThreads * (int)gridDim.x)
            L.vec[(size_t)V_U * L.ld + i] = 0.f;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *L.st = S;
        *A.active_after = S.phase != PH_DONE ? 1 : 0;
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

static size_t solo_smem(int ld, int grid) { return (grid == 1 ? 6 : 2) * (size_t)ld * sizeof(float); }

cudaError_t prepare_solo(int ld)
{
    const size_t smem = solo_smem(ld, 1);
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(solo_lane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// every CTA must be resident: a cooperative launch fails instead of starting a grid that
// could not be
cudaError_t launch_solo(const SoloArgs& a, int ld, cudaStream_t s)
{
    SoloArgs args = a;
    void* params[] = {&args};
    return cudaLaunchCooperativeKernel((const void*)solo_lane_kernel, dim3((unsigned)a.grid), dim3(kThreads), params,
                                       solo_smem(ld, a.grid), s);
}

}  // namespace ubqp
