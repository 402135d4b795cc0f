// Phase A on the 5th-generation tensor cores: the matvecs of all starts of an instance as
// one contraction  D = Q_off * U^T  (Q_off in BF16, U = the lanes' inputs as BF16 hi + lo
// rows, FP32 accumulation in TMEM), for the batched-restart and ragged paths.
//
// Tiling.  One CTA owns a 128-row M tile of one instance, an N tile of up to 128 lanes and
// a slice of the K dimension; the S CTAs of a thread-block cluster share the M/N tile and
// split K.  A (128 x 64) and B (N x 64) k-blocks arrive by TMA in 128-byte-swizzled tiles
// into a shared-memory ring, the lanes' hi rows and lo rows back to back; one thread issues
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, K = 16 per instruction, N = twice the
// tile's lanes, so one MMA covers both terms) and tcgen05.commit frees ring slots.  The
// accumulators are then read with tcgen05.ld, parked in shared memory and summed across the
// cluster through distributed shared memory; every CTA finishes a subset of the lanes with the
// per-row epilogue of the lane's phase, whose operand rows each warp has meanwhile copied
// (cp.async, a few lanes ahead) into slots of the freed ring after the accumulators.
//
// Every mbarrier wait is bounded (2 s of globaltimer); on expiry the CTA records an error,
// stops issuing work, still passes every cluster barrier and frees its TMEM.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>
#include <cstring>

#include "../../include/ubqp.h"
#include "lane_update.cuh"
#include "ubqp_engine.cuh"
#include "ubqp_tc.cuh"

namespace cg = cooperative_groups;

namespace ubqp {

namespace {

constexpr int kTcThreads = 256;       // 8 warps: TMA producer, MMA issuer, then all 8 drain TMEM / run the epilogue
constexpr uint64_t kWaitNs = 2000000000ull;
// split-K kernel epilogue: each warp stages the operand rows of its next kEpiDepth lanes in
// shared memory (slots of kEpiSlot floats = 7 vectors x 128 rows, after the accumulators)
constexpr int kEpiDepth = 3;
constexpr int kEpiSlot = 7 * 128;
constexpr size_t kEpiSlotBytes = (size_t)(kTcThreads / 32) * kEpiDepth * kEpiSlot * 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte asynchronous copy global -> shared (L2 only); groups complete in commit order
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bounded parity wait: false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    const uint64_t t0 = globaltimer();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major operand in 128-byte-swizzled 8-row atoms
// (rows of 128 bytes, 1024 bytes between 8-row groups), descriptor version 1
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (not used by swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Accumulator layout.  The hi and lo rows of the inputs sit back to back in shared memory,
// so one MMA with N = 2 bn covers both terms: columns [0, bn) of its accumulator collect the
// hi products, [bn, 2 bn) the lo products.  Each MMA instruction costs a similar time
// whatever its N up to 256 (measured: ~155 cycles for N = 16 and ~170 for N = 128), so fewer,
// wider instructions are what raises throughput.  The k-steps of a tile are also dealt
// round-robin to tc_chains_k(bn) accumulators (chain c at column offset c * w, w = 2 bn or bn)
// so that consecutive MMAs do not all accumulate into one place.  The drain adds, for each
// column, the hi parts of the chains in ascending order, then the lo parts; both kernels use
// this layout, so a tile's sums do not depend on which kernel computed it.
__host__ __device__ constexpr int tc_chains_k(int bn) { return bn <= 32 ? 4 : (bn <= 64 ? 2 : 1); }

// 16 consecutive output columns of this thread's TMEM lane, summed over terms and chains
__device__ __forceinline__ void tmem_ld16_sum(uint32_t taddr, int bn, bool two, float* v)
{
    const int nk = tc_chains_k(bn), w = two ? 2 * bn : bn;
    tmem_ld16(taddr, v);
    for (int t = 0; t < (two ? 2 : 1); ++t)
        for (int c = (t == 0 ? 1 : 0); c < nk; ++c) {
            float u[16];
            tmem_ld16(taddr + (uint32_t)(c * w + t * bn), u);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += u[i];
        }
}

// warp-level reduction of one lane's accumulator into its partial record (lane 0 writes)
__device__ __forceinline__ void warp_reduce_write(Acc& a, int ph, Partial* out, bool has_f)
{
    acc_shfl_reduce(a, ph, has_f);
    if ((threadIdx.x & 31) == 0) {
        Partial P;
#pragma unroll
        for (int t = 0; t < 12; ++t) P.s[t] = a.s[t];
#pragma unroll
        for (int t = 0; t < 6; ++t) P.m[t] = a.m[t];
        P.f = has_f ? a.f : 0.0;
        *out = P;
    }
}

}  // namespace

// Per-row epilogue of one lane of an M tile (rows mt*128 + lane + 32 j, j < 4, values vv
// from the contraction) and its partial record part[mt], by one warp.  The gradient step and
// the eigen-solver steps (the steps that dominate a solve) are split into loading their
// operands and finishing, so that the lane loops can load the next lane's operands while they
// finish the current one; the arithmetic and its order are those of row_epilogue.
//   gradient step (Alg. 2, g^k): x, d - p, tsum, x_prev, g_{k-1}, |Q'_off| row sum;
//   eigen-solver steps (Lemma 3.1, LOBPCG on Z^-1/2 Qbar_II Z^-1/2): D, w, d - p and, for an
//   iteration, the basis vectors x, Ax, p, Ap.
struct EpiOps {
    float v[7][4];
};

__device__ __forceinline__ bool epi_ops_phase(int ph) { return ph == PH_INNER || ph == PH_LOB || ph == PH_LOB_INIT; }

__device__ __forceinline__ void tc_epi_load(const float* vec, const float* tsum, const float* oabs, int ph, int ld, int n,
                                            int mt, int lane, EpiOps& o)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = min(mt * 128 + lane + 32 * j, n - 1);
        if (ph == PH_INNER) {
            o.v[0][j] = vec[V_X * ld + i];
            o.v[1][j] = vec[V_DMP * ld + i];
            o.v[2][j] = tsum[i];
            o.v[3][j] = vec[V_XPREV * ld + i];
            o.v[4][j] = vec[V_G * ld + i];
            o.v[5][j] = oabs[i];
        } else {
            o.v[0][j] = vec[V_D * ld + i];
            o.v[1][j] = vec[(ph == PH_LOB_INIT ? V_LX : V_LW) * ld + i];
            o.v[2][j] = vec[V_DMP * ld + i];
            if (ph == PH_LOB) {
                o.v[3][j] = vec[V_LX * ld + i];
                o.v[4][j] = vec[V_LAX * ld + i];
                o.v[5][j] = vec[V_LP * ld + i];
                o.v[6][j] = vec[V_LAP * ld + i];
            }
        }
    }
}

__device__ __forceinline__ void tc_epi_finish(float* vec, Partial* part, int ph, int ld, int n, int mt, int k,
                                              const float (&vv)[4], int lane, const EpiOps& o)
{
    Acc a;
    a.zero();
    if (ph == PH_INNER) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = mt * 128 + lane + 32 * j;
            if (i >= n) continue;
            const float x = o.v[0][j], dmp = o.v[1][j];
            const float g = fmaf(dmp, 2.f * x - 1.f, fmaf(2.f, vv[j], o.v[2][j]));
            if (k >= 1) {
                const float sj = x - o.v[3][j], yj = g - o.v[4][j];
                csum_add(a.s[0], sj * sj);
                csum_add(a.s[1], sj * yj);
                csum_add(a.s[2], yj * yj);
            } else {
                a.m[1] = fmaxf(a.m[1], fabsf(dmp));
                a.m[2] = fmaxf(a.m[2], fabsf(vec[V_BBAR * ld + i]));
                a.m[3] = fmaxf(a.m[3], o.v[5][j] + fabsf(dmp));
            }
            vec[V_G * ld + i] = g;
            const float viol = (x > 0.f && x < 1.f) ? fabsf(g) : (x <= 0.f ? fmaxf(-g, 0.f) : fmaxf(g, 0.f));
            a.m[0] = fmaxf(a.m[0], viol);
        }
        warp_reduce_write(a, PH_INNER, part + mt, false);
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = mt * 128 + lane + 32 * j;
        if (i >= n) continue;
        const float Dz = o.v[0][j], w = o.v[1][j];
        float aw = 0.f;
        if (Dz != 0.f) aw = Dz * fmaf(o.v[2][j], Dz * w, vv[j]);
        vec[V_W * ld + i] = aw;
        if (ph == PH_LOB_INIT) {
            csum_add(a.s[0], w * aw);
            csum_add(a.s[1], w * w);
        } else {
            const float x = o.v[3][j], ax = o.v[4][j], p = o.v[5][j], ap = o.v[6][j];
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
    }
    warp_reduce_write(a, ph, part + mt, false);
}

// the fields of a lane's descriptor that the prefetched epilogues use
struct LaneEpi {
    float* vec;
    const float* tsum;
    const float* oabs;
    Partial* part;
};

// One warp copies a lane's operand rows ms .. ms + 127 (512 bytes per vector) into a slot:
// gradient step x, d - p, x_prev, g_{k-1}; eigen-solver steps D, w, d - p (and x, Ax, p, Ap).
__device__ __forceinline__ void tc_epi_copy(const float* vec, int ph, int ld, int ms, float* slot, int lane)
{
    int vs[7];
    int nv;
    if (ph == PH_INNER) {
        vs[0] = V_X; vs[1] = V_DMP; vs[2] = V_XPREV; vs[3] = V_G;
        nv = 4;
    } else {
        vs[0] = V_D; vs[1] = ph == PH_LOB_INIT ? V_LX : V_LW; vs[2] = V_DMP;
        vs[3] = V_LX; vs[4] = V_LAX; vs[5] = V_LP; vs[6] = V_LAP;
        nv = ph == PH_LOB_INIT ? 3 : 7;
    }
#pragma unroll
    for (int a = 0; a < 7; ++a)
        if (a < nv) cp_async16(slot + a * 128 + 4 * lane, vec + (size_t)vs[a] * ld + ms + 4 * lane);
}

// the operands of rows lane + 32 j from a slot (and the instance's tsum and |Q'_off| row sums
// of the tile, `inst`), in the order tc_epi_load gives them
__device__ __forceinline__ void tc_epi_from_slot(const float* slot, const float (*inst)[128], int ph, int lane,
                                                 EpiOps& o)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = lane + 32 * j;
        if (ph == PH_INNER) {
            o.v[0][j] = slot[r];
            o.v[1][j] = slot[128 + r];
            o.v[2][j] = inst[0][r];
            o.v[3][j] = slot[256 + r];
            o.v[4][j] = slot[384 + r];
            o.v[5][j] = inst[1][r];
        } else {
#pragma unroll
            for (int a = 0; a < 7; ++a) o.v[a][j] = slot[a * 128 + r];
        }
    }
}

// any phase; `pre` holds the operands when the caller already loaded them (epi_ops_phase)
__device__ __forceinline__ void tc_lane_epilogue(const TcArgs& A, const TcInst& I, int mt, int r, int ph, int k,
                                                 const float (&vv)[4], int lane, const EpiOps* pre)
{
    const LaneDev& L = A.lanes[I.lane0 + r];
    if (epi_ops_phase(ph)) {
        if (pre) {
            tc_epi_finish(L.vec, L.part, ph, I.ld, I.n, mt, k, vv, lane, *pre);
        } else {
            EpiOps o;
            tc_epi_load(L.vec, L.tsum, L.oabs, ph, I.ld, I.n, mt, lane, o);
            tc_epi_finish(L.vec, L.part, ph, I.ld, I.n, mt, k, vv, lane, o);
        }
        return;
    }
    Acc a;
    a.zero();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = mt * 128 + lane + 32 * j;
        if (i < I.n) row_epilogue(L, ph, k, i, (double)vv[j], a, A.P.tau_z);
    }
    warp_reduce_write(a, ph, L.part + mt, ph == PH_EVAL);
}

// Fused update: after a warp has written lane L's partial for one M tile it counts itself in;
// the warp that completes the lane's count (all its M tiles done, so no CTA of this launch
// still reads the lane's inputs) runs the lane's update.
__device__ __forceinline__ void tc_fused_count(const TcArgs& A, const LaneDev& L, WarpUpd& W)
{
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if ((threadIdx.x & 31) == 0) last = atomicAdd(L.counter, 1u) == (unsigned)(L.nblk - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
        __threadfence();
        if ((threadIdx.x & 31) == 0) *L.counter = 0u;
        __syncwarp();
        warp_lane_update(L, A.P, W, A.active_count);
        // the inputs written here are read by the next step's TMA loads (async proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
}

// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1) phase_a_tc_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned ring
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full_bar[kTcMaxStages], empty_bar[kTcMaxStages], accum_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_inst, s_mt, s_nt, s_skip;
    __shared__ int s_fail;
    __shared__ WarpUpd s_upd[kTcThreads / 32];

    cg::cluster_group cluster = cg::this_cluster();
    const int S = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // ---- which tile: clusters are consecutive blocks
    if (threadIdx.x == 0) {
        const int c = blockIdx.x / S;
        int lo = 0, hi = A.ninst - 1;   // last instance whose first cluster index <= c
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A.inst[mid].cluster0 <= c) lo = mid; else hi = mid - 1;
        }
        const TcInst& I = A.inst[lo];
        const int local = c - I.cluster0;
        s_inst = lo;
        s_mt = local / I.n_tiles;
        s_nt = local % I.n_tiles;
        s_fail = 0;
        // a tile whose lanes are all finished is skipped by every CTA of the cluster
        int alive = A.raw ? 1 : 0;
        if (!A.raw && I.nt_active) {
            alive = I.nt_active[s_nt] > 0;
        } else if (!A.raw) {
            const int r0 = s_nt * I.bn, r1 = min(I.R, r0 + I.bn);
            for (int r = r0; r < r1 && !alive; ++r) alive = A.lanes[I.lane0 + r].st->phase != PH_DONE;
        }
        s_skip = !alive;
    }
    __syncthreads();
    const TcInst& I = A.inst[s_inst];
    const int mt = s_mt, nt = s_nt;
    const int BN = I.bn;
    const bool two = I.two_terms != 0;
    const int kb_total = I.ld / 64;
    const int kb0 = (int)((int64_t)kb_total * rank / S), kb1 = (int)((int64_t)kb_total * (rank + 1) / S);
    const int nkb = kb1 - kb0;
    const uint32_t a_bytes = 128 * 128, b_bytes = (uint32_t)BN * 128;
    const uint32_t stage_bytes = a_bytes + b_bytes * (two ? 2u : 1u);
    const int NS = A.stages;

    if (!s_skip) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < NS; ++s) {
                mbar_init(&full_bar[s], 1);
                mbar_init(&empty_bar[s], 1);
            }
            mbar_init(&accum_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 1) tmem_alloc(&tmem_base, (uint32_t)A.tmem_cols);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();

    // this CTA's share of the tile's lanes for the epilogue; warps 2.. (idle while warps 0 and 1
    // run the main loop) read their states and descriptor fields now (neither changes during
    // the launch)
    __shared__ int s_ph[kTcMaxBn], s_k[kTcMaxBn];
    __shared__ LaneEpi s_epi[kTcMaxBn];
    __shared__ __align__(16) float s_rows[2][128];   // tsum and |Q'_off| row sums of the tile's rows
    const int nreal = min(BN, I.R - nt * BN);
    const int c0 = (int)((int64_t)nreal * rank / S), c1 = (int)((int64_t)nreal * (rank + 1) / S);
    if (!s_skip && !A.raw && warp >= 2)
        for (int c = c0 + (int)threadIdx.x - 64; c < c1; c += kTcThreads - 64) {
            const LaneDev& Ld = A.lanes[I.lane0 + nt * BN + c];
            const LaneState* st = Ld.st;
            s_ph[c - c0] = st->phase;
            s_k[c - c0] = st->k;
            s_epi[c - c0] = LaneEpi{Ld.vec, Ld.tsum, Ld.oabs, Ld.part};
        }

    if (!s_skip && nkb > 0) {
        const uint32_t tmem = tmem_base;
        if (warp == 0 && lane == 0) {
            // TMA producer
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % NS;
                if (kb >= NS && !mbar_wait(&empty_bar[s], (uint32_t)((kb / NS - 1) & 1))) { s_fail = 1; break; }
                issued = kb + 1;
                unsigned char* st = ring + (size_t)s * stage_bytes;
                mbar_expect_tx(&full_bar[s], stage_bytes);
                const int kx = (kb0 + kb) * 64;
                tma_load_2d(st, &I.tmA, &full_bar[s], 0, (mt * kb_total + kb0 + kb) * 128);
                tma_load_2d(st + a_bytes, &I.tmBhi, &full_bar[s], kx, nt * BN);
                if (two) tma_load_2d(st + a_bytes + b_bytes, &I.tmBlo, &full_bar[s], kx, nt * BN);
            }
            if (s_fail) {
                // a wait ran out: let every copy already issued land before the ring is reused
                for (int kb = (issued > NS ? issued - NS : 0); kb < issued; ++kb)
                    mbar_wait(&full_bar[kb % NS], (uint32_t)((kb / NS) & 1));
            }
        } else if (warp == 1 && lane == 0) {
            // MMA issuer: 4 K-steps of 16 per 64-wide k-block, both terms in one MMA of N = 2 BN
            const uint32_t idesc = idesc_bf16(128, two ? 2 * BN : BN);
            const int NK = tc_chains_k(BN), W = two ? 2 * BN : BN;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % NS;
                if (!mbar_wait(&full_bar[s], (uint32_t)((kb / NS) & 1))) { s_fail = 1; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(ring + (size_t)s * stage_bytes);
                const uint32_t sb = sa + a_bytes;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int ks = kb * 4 + k, ck = ks % NK;
                    umma_bf16(tmem + (uint32_t)(ck * W), sdesc_sw128(sa + k * 32), sdesc_sw128(sb + k * 32), idesc,
                              ks >= NK ? 1u : 0u);
                }
                umma_commit(&empty_bar[s]);
            }
            umma_commit(&accum_bar);
        }
        __syncwarp();
    }
    __syncthreads();

    // ---- accumulators -> shared memory P[col][row] (the ring is free once accum_bar fired).
    // One thread waits on the barrier; the rest sleep at __syncthreads.
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = (!s_skip && nkb > 0) ? (!s_fail && mbar_wait(&accum_bar, 0u)) : 1;
    __syncthreads();
    float* P = reinterpret_cast<float*>(ring);
    // operand slots after the accumulators (the ring is free now); warp w's lanes are
    // c0 + w + 8 t, lane t in slot t mod kEpiDepth, one copy group per lane
    float* slots = P + 128 * A.max_bn + (size_t)warp * kEpiDepth * kEpiSlot;
    auto epi_issue = [&](int t) {
        const int c = c0 + warp + (kTcThreads / 32) * t;
        if (!A.raw && c < c1 && epi_ops_phase(s_ph[c - c0]))
            tc_epi_copy(s_epi[c - c0].vec, s_ph[c - c0], I.ld, mt * 128, slots + (t % kEpiDepth) * kEpiSlot, lane);
        cp_async_commit();
    };
    if (!s_skip) {
        if (!A.raw && threadIdx.x < 64) {
            // the instance's vectors, through any of the CTA's lanes
            if (c0 < c1) {
                const float* src = threadIdx.x < 32 ? s_epi[0].tsum : s_epi[0].oabs;
                cp_async16(&s_rows[threadIdx.x >> 5][4 * lane], src + mt * 128 + 4 * lane);
            }
            cp_async_commit();
        }
#pragma unroll
        for (int t = 0; t < kEpiDepth; ++t) epi_issue(t);
    }
    if (!s_skip) {
        const bool have = nkb > 0 && s_ok;
        if (nkb > 0) tc_fence_after();
        const int row = (warp & 3) * 32 + lane;   // TMEM lanes reachable by this warp
        for (int q = warp >> 2; q < BN / 16; q += 2) {   // 16-column chunks split over the two warpgroups
            float v[16];
            if (have) {
                tmem_ld16_sum(tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(q * 16), BN, two, v);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) P[(q * 16 + i) * 128 + row] = v[i];
        }
        if (!s_ok && threadIdx.x == 0) {
            s_fail = 1;
            if (A.err) atomicExch(A.err, 1);
        }
        tc_fence_before();
    }
    cluster.sync();

    // ---- sum the cluster's partial accumulators and run the epilogue for this CTA's lanes
    if (!s_skip) {
        if (A.flops && rank == 0 && threadIdx.x == 0)   // 2 n flops per (row, lane), single term
            atomicAdd(A.flops, 2ull * (unsigned long long)min(128, I.n - mt * 128) * (unsigned long long)I.n *
                                   (unsigned long long)nreal);
        if (A.P.bytes && rank == 0 && threadIdx.x == 0) {
            // algorithmic bytes: the M tile's rows of Q_off once per step (BF16, charged to the
            // first N tile) and the starts' inputs once (charged to the first M tile)
            unsigned long long by = 0;
            if (nt == 0) by += 2ull * (unsigned long long)min(128, I.n - mt * 128) * (unsigned long long)I.n;
            if (mt == 0) by += 2ull * (two ? 2ull : 1ull) * (unsigned long long)nreal * (unsigned long long)I.n;
            atomicAdd(A.P.bytes, by);
        }
        if (!A.raw && threadIdx.x < 64) cp_async_wait<kEpiDepth>();   // the tile's tsum and row sums
        __syncthreads();
        float* peers[kTcMaxCluster];
        for (int q = 0; q < S; ++q) peers[q] = cluster.map_shared_rank(P, q);
        // lanes c0 + warp, + 8, ...: the operands come from the warp's slots; the next lane's
        // cluster partials (every rank's value of its four rows, summed in rank order when its
        // turn comes) load while this one finishes
        float pcur[kTcMaxCluster][4], pnxt[kTcMaxCluster][4];
        auto load_parts = [&](int c, float (&pv)[kTcMaxCluster][4]) {
#pragma unroll
            for (int q = 0; q < kTcMaxCluster; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (q < S) pv[q][j] = peers[q][c * 128 + lane + 32 * j];
        };
        if (c0 + warp < c1) load_parts(c0 + warp, pcur);
        for (int c = c0 + warp, t = 0; c < c1; c += kTcThreads / 32, ++t) {
            const int r = nt * BN + c;  // restart index within the instance
            const int cn = c + kTcThreads / 32;
            if (cn < c1) load_parts(cn, pnxt);
            const int ph = A.raw ? PH_DONE : s_ph[c - c0];
            const bool staged = epi_ops_phase(ph);
            EpiOps cur;
            cp_async_wait<kEpiDepth - 1>();   // lane t's group
            __syncwarp();
            if (staged) tc_epi_from_slot(slots + (t % kEpiDepth) * kEpiSlot, s_rows, ph, lane, cur);
            __syncwarp();                     // the slot is read: it takes lane t + kEpiDepth
            epi_issue(t + kEpiDepth);
            float vv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < kTcMaxCluster; ++q)
                    if (q < S) acc += pcur[q][j];
                vv[j] = acc;
            }
            if (A.raw) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = mt * 128 + lane + 32 * j;
                    if (i < I.n) A.raw[(size_t)r * I.ld + i] = vv[j];
                }
            } else if (ph != PH_DONE) {
                if (staged) tc_epi_finish(s_epi[c - c0].vec, s_epi[c - c0].part, ph, I.ld, I.n, mt, s_k[c - c0], vv, lane, cur);
                else tc_lane_epilogue(A, I, mt, r, ph, s_k[c - c0], vv, lane, nullptr);
                if (A.fuse) tc_fused_count(A, A.lanes[I.lane0 + r], s_upd[warp]);
            }
#pragma unroll
            for (int q = 0; q < kTcMaxCluster; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j) pcur[q][j] = pnxt[q][j];
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // no copy into this CTA's slots outstanding
    cluster.sync();  // peers' shared memory stays alive until every CTA has read it

    if (!s_skip) {
        __syncthreads();
        if (warp == 1) {
            tc_fence_after();
            tmem_dealloc(tmem_base, (uint32_t)A.tmem_cols);
        }
    }
}

// ---------------------------------------------------------------------------------
// Persistent form for launches with many tiles (the ragged batch): no split-K, one CTA per
// SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... and overlaps the epilogue of
// one tile with the contraction of the next.
//
// Roles: warp 0 (one thread) keeps the TMA ring full across tile boundaries; warp 1 (one
// thread) issues the MMAs of each tile into one of two TMEM accumulators (columns
// buf * max_bn), waiting until the epilogue has drained that buffer; warps 4..7 drain the
// finished accumulator into shared memory (each warp reaches TMEM lanes 32 (w mod 4) ..)
// and release it; warps 2..7 then run the per-row epilogue of the tile's lanes.  All roles
// walk the same tile list and skip the same finished tiles (lane states do not change
// during the launch).  Waits are bounded; after a failure every role stops working but the
// epilogue warps keep their named barriers matched, and the CTA lets issued copies and
// MMAs complete before it frees shared memory and TMEM.
struct TcTile {
    int inst, mt, nt, kb;
    bool alive;
};

__device__ __forceinline__ TcTile tcp_tile(const TcArgs& A, int t)
{
    int lo = 0, hi = A.ninst - 1;   // last instance whose first tile index <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.inst[mid].cluster0 <= t) lo = mid; else hi = mid - 1;
    }
    const TcInst& I = A.inst[lo];
    const int local = t - I.cluster0;
    TcTile T;
    T.inst = lo;
    T.mt = local / I.n_tiles;
    T.nt = local % I.n_tiles;
    T.kb = I.ld / 64;
    T.alive = A.raw != nullptr;
    if (!T.alive && I.nt_active) {
        T.alive = I.nt_active[T.nt] > 0;
    } else if (!T.alive) {
        const int r0 = T.nt * I.bn, r1 = min(I.R, r0 + I.bn);
        for (int r = r0; r < r1 && !T.alive; ++r) T.alive = A.lanes[I.lane0 + r].st->phase != PH_DONE;
    }
    return T;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epi_bar_sync() { asm volatile("bar.sync 1, 192;" ::: "memory"); }

__device__ __forceinline__ int vload(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

__global__ void __launch_bounds__(kTcThreads, 1) phase_a_tcp_kernel(TcArgs A, int ntiles)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS = A.stages;
    const uint32_t stage_max = 128u * 128u + (uint32_t)A.max_bn * 128u * (A.two_any ? 2u : 1u);
    float* P = reinterpret_cast<float*>(ring + (size_t)NS * stage_max);
    __shared__ uint64_t full_bar[kTcpMaxStages], empty_bar[kTcpMaxStages], accf_bar[2], acce_bar[2], fin_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ long long s_issued;
    __shared__ WarpUpd s_upd[kTcThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t col_stride = A.two_any ? 256u : 128u;   // one accumulator buffer: terms x chains x bn <= this

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], 4);   // one arrival per draining warp
        }
        mbar_init(&fin_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_issued = 0;
    }
    if (warp == 1) tmem_alloc(&tmem_base, (uint32_t)A.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {   // ---- TMA producer
            long long pos = 0;
            for (int t = blockIdx.x; t < ntiles && !vload(&s_fail); t += gridDim.x) {
                const TcTile T = tcp_tile(A, t);
                if (!T.alive) continue;
                const TcInst& I = A.inst[T.inst];
                const bool two = I.two_terms != 0;
                const uint32_t a_bytes = 128u * 128u, b_bytes = (uint32_t)I.bn * 128u;
                const uint32_t sb = a_bytes + b_bytes * (two ? 2u : 1u);
                for (int kb = 0; kb < T.kb; ++kb, ++pos) {
                    const int s = (int)(pos % NS);
                    const long long use = pos / NS;
                    if (use > 0 && !mbar_wait(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
                        s_fail = 1;
                        break;
                    }
                    unsigned char* st = ring + (size_t)s * stage_max;
                    mbar_expect_tx(&full_bar[s], sb);
                    tma_load_2d(st, &I.tmA, &full_bar[s], 0, (T.mt * T.kb + kb) * 128);
                    tma_load_2d(st + a_bytes, &I.tmBhi, &full_bar[s], kb * 64, T.nt * I.bn);
                    if (two) tma_load_2d(st + a_bytes + b_bytes, &I.tmBlo, &full_bar[s], kb * 64, T.nt * I.bn);
                    s_issued = pos + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---- MMA issuer
            long long pos = 0;
            int j = 0;
            for (int t = blockIdx.x; t < ntiles && !vload(&s_fail); t += gridDim.x) {
                const TcTile T = tcp_tile(A, t);
                if (!T.alive) continue;
                const TcInst& I = A.inst[T.inst];
                const bool two = I.two_terms != 0;
                const uint32_t a_bytes = 128u * 128u;
                const int buf = j & 1, use_b = j >> 1;
                if (use_b > 0 && !mbar_wait(&acce_bar[buf], (uint32_t)((use_b - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)buf * col_stride;
                const uint32_t idesc = idesc_bf16(128, two ? 2 * I.bn : I.bn);
                const int NK = tc_chains_k(I.bn), W = two ? 2 * I.bn : I.bn;
                bool ok = true;
                for (int kb = 0; kb < T.kb; ++kb, ++pos) {
                    const int s = (int)(pos % NS);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((pos / NS) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(ring + (size_t)s * stage_max);
                    const uint32_t sbh = sa + a_bytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int ks = kb * 4 + k, ck = ks % NK;
                        umma_bf16(d + (uint32_t)(ck * W), sdesc_sw128(sa + k * 32), sdesc_sw128(sbh + k * 32), idesc,
                                  ks >= NK ? 1u : 0u);
                    }
                    umma_commit(&empty_bar[s]);
                }
                if (!ok) {
                    s_fail = 1;
                    break;
                }
                umma_commit(&accf_bar[buf]);
                ++j;
            }
            // every MMA issued has completed before TMEM is released
            if (pos > 0) {
                umma_commit(&fin_bar);
                mbar_wait(&fin_bar, 0u);
            }
        }
    } else {
        // ---- warps 2..7: epilogue; warps 4..7 first drain TMEM into P[col][row]
        const bool drain = warp >= 4;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TcTile T = tcp_tile(A, t);
            if (!T.alive) continue;
            const TcInst& I = A.inst[T.inst];
            const int buf = j & 1, use_b = j >> 1;
            if (drain) {
                int ok = 0;
                if (lane == 0) ok = !vload(&s_fail) && mbar_wait(&accf_bar[buf], (uint32_t)(use_b & 1));
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok && lane == 0) s_fail = 1;
                tc_fence_after();
                const int row = (warp & 3) * 32 + lane;
                for (int q = 0; q < I.bn / 16; ++q) {
                    float v[16];
                    if (ok) {
                        tmem_ld16_sum(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)buf * col_stride +
                                          (uint32_t)(q * 16),
                                      I.bn, I.two_terms != 0, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) P[(q * 16 + i) * 128 + row] = v[i];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0 && ok) mbar_arrive(&acce_bar[buf]);
            }
            epi_bar_sync();   // P holds this tile's products
            if (!vload(&s_fail)) {
                const int nreal = min(I.bn, I.R - T.nt * I.bn);
                if (warp == 2 && lane == 0) {
                    const unsigned long long rows = (unsigned long long)min(128, I.n - T.mt * 128);
                    if (A.flops) atomicAdd(A.flops, 2ull * rows * (unsigned long long)I.n * (unsigned long long)nreal);
                    if (A.P.bytes) {
                        unsigned long long by = 0;
                        if (T.nt == 0) by += 2ull * rows * (unsigned long long)I.n;
                        if (T.mt == 0)
                            by += 2ull * (I.two_terms ? 2ull : 1ull) * (unsigned long long)nreal * (unsigned long long)I.n;
                        atomicAdd(A.P.bytes, by);
                    }
                }
                // lanes warp - 2, + 6, ...: the next lane's operands load while this one finishes
                EpiOps cur, nxt;
                int cur_ph = PH_DONE, cur_k = 0;
                auto lane_at = [&](int c, EpiOps& o, int& ph, int& k) {
                    ph = PH_DONE;
                    if (A.raw || c >= nreal) return;
                    const LaneDev& L = A.lanes[I.lane0 + T.nt * I.bn + c];
                    const LaneState* st = L.st;
                    ph = st->phase;
                    k = st->k;
                    if (epi_ops_phase(ph)) tc_epi_load(L.vec, L.tsum, L.oabs, ph, I.ld, I.n, T.mt, lane, o);
                };
                lane_at(warp - 2, cur, cur_ph, cur_k);
                for (int c = warp - 2; c < nreal; c += 6) {
                    const int r = T.nt * I.bn + c;
                    int nxt_ph, nxt_k = 0;
                    lane_at(c + 6, nxt, nxt_ph, nxt_k);
                    float vv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) vv[q] = P[c * 128 + lane + 32 * q];
                    if (A.raw) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int i = T.mt * 128 + lane + 32 * q;
                            if (i < I.n) A.raw[(size_t)r * I.ld + i] = vv[q];
                        }
                    } else if (cur_ph != PH_DONE) {
                        tc_lane_epilogue(A, I, T.mt, r, cur_ph, cur_k, vv, lane, epi_ops_phase(cur_ph) ? &cur : nullptr);
                        if (A.fuse) tc_fused_count(A, A.lanes[I.lane0 + r], s_upd[warp]);
                    }
                    cur = nxt;
                    cur_ph = nxt_ph;
                    cur_k = nxt_k;
                }
            }
            epi_bar_sync();   // P may be overwritten
            ++j;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) {
        if (A.err) atomicExch(A.err, 1);
        // copies already issued land before the ring's shared memory goes away
        const long long iss = s_issued;
        for (long long q = (iss > NS ? iss - NS : 0); q < iss; ++q)
            mbar_wait(&full_bar[q % NS], (uint32_t)((q / NS) & 1));
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)A.tmem_cols);
    }
}

// ---------------------------------------------------------------------------------
static int pow2_at_least(int v)
{
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

size_t tc_smem_bytes(int bn, bool two, int stages)
{
    const size_t stage = 128 * 128 + (size_t)bn * 128 * (two ? 2 : 1);
    // reused for the accumulators and the epilogue's operand slots
    const size_t ring = std::max(stage * stages, (size_t)bn * 128 * 4 + kEpiSlotBytes);
    return ring + 1024;  // alignment slack
}

int tc_pick_stages(int bn, bool two)
{
    const size_t stage = 128 * 128 + (size_t)bn * 128 * (two ? 2 : 1);
    int s = (int)((200 * 1024) / stage);
    if (s > kTcMaxStages) s = kTcMaxStages;
    if (s < 2) s = 2;
    return s;
}

// persistent kernel: ring of `stages` slots of the largest stage, then P (max_bn x 128 FP32)
size_t tcp_smem_bytes(int bn, bool two, int stages)
{
    const size_t stage = 128 * 128 + (size_t)bn * 128 * (two ? 2 : 1);
    return stage * stages + (size_t)bn * 128 * 4 + 1024;
}

int tcp_pick_stages(int bn, bool two)
{
    const size_t stage = 128 * 128 + (size_t)bn * 128 * (two ? 2 : 1);
    const size_t room = 210 * 1024 - (size_t)bn * 128 * 4 - 1024;
    int s = (int)(room / stage);
    if (s > kTcpMaxStages) s = kTcpMaxStages;
    return s;   // < 2: the persistent kernel does not fit this tile width
}

// two accumulator buffers of terms x chains x bn <= 128 per term columns each
int tcp_tmem_cols(bool two) { return two ? 512 : 256; }

// one CTA per SM (as many as fit), never more than the tiles
int tcp_grid(const TcArgs& a, int ntiles)
{
    const size_t smem = tcp_smem_bytes(a.max_bn, a.two_any != 0, a.stages);
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(phase_a_tcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, phase_a_tcp_kernel, kTcThreads, smem) != cudaSuccess ||
        per < 1) {
        cudaGetLastError();
        per = 1;
    }
    const int g = sms * per;
    return ntiles < g ? ntiles : g;
}

cudaError_t tcp_launch(const TcArgs& a, int ntiles, int grid, cudaStream_t st)
{
    const size_t smem = tcp_smem_bytes(a.max_bn, a.two_any != 0, a.stages);
    cudaError_t e = cudaFuncSetAttribute(phase_a_tcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    phase_a_tcp_kernel<<<grid, kTcThreads, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

cudaError_t tc_launch(const TcArgs& a, int total_clusters, int S, cudaStream_t st)
{
    size_t smem = tc_smem_bytes(a.max_bn, a.two_any != 0, a.stages);
    cudaError_t e = cudaFuncSetAttribute(phase_a_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(total_clusters * S), 1, 1);
    cfg.blockDim = dim3(kTcThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, phase_a_tc_kernel, a);
}

int tc_max_active_clusters(int bn, bool two, int stages, int S)
{
    size_t smem = tc_smem_bytes(bn, two, stages);
    if (cudaFuncSetAttribute(phase_a_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(S * 64), 1, 1);
    cfg.blockDim = dim3(kTcThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, phase_a_tc_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int tc_tmem_cols(int bn, bool two) { return pow2_at_least((two ? 2 : 1) * tc_chains_k(bn) * bn); }

int tc_pick_cluster(int tiles, int kb_min, int bn, bool two, int stages, int num_sms)
{
    int best = 1;
    for (int S = 1; S <= 8; ++S) {
        if (tiles * S > num_sms) break;
        if (kb_min / S < 2 && S > 1) break;
        if (tc_max_active_clusters(bn, two, stages, S) < tiles) continue;
        best = S;
    }
    return best;
}

// 2-D BF16 tensor map over a row-major [rows][cols] array, box 64 (cols) x box_rows
// cuTensorMapEncodeTiled is a driver entry point; resolving it through the runtime keeps
// the library loadable (for its CPU-side checks) on machines without a driver
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

CUresult tc_encode_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return CUDA_ERROR_NOT_FOUND;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace ubqp

// =====================================================================================
// Test entry: D = A * (B_hi + B_lo)^T through the tensor-core kernel, raw output.
using namespace ubqp;

extern "C" int ubqp_tc_matmul_probe(const uint16_t* A, const uint16_t* Bhi, const uint16_t* Blo, int64_t n,
                                    int64_t R, int32_t cluster, float* D_out)
{
    if (!A || !Bhi || !D_out || n < 1 || n > 32768 || R < 1 || R > 1024 || cluster < -1 || cluster > 8)
        return UBQP_EINVAL;
    const int ld = (int)((n + 127) / 128 * 128);
    const int rpad = (int)((R + 15) / 16 * 16);
    const int bn = rpad < kTcMaxBn ? rpad : kTcMaxBn;
    const int n_tiles = (rpad + bn - 1) / bn;
    const int rows_b = n_tiles * bn;
    const bool two = Blo != nullptr;
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) return UBQP_ECUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t bytesA = (size_t)ld * ld * 2, bytesB = (size_t)rows_b * ld * 2, bytesD = (size_t)R * ld * 4;
    char* buf = nullptr;
    const size_t off_bhi = (bytesA + 255) / 256 * 256;
    const size_t off_blo = off_bhi + (bytesB + 255) / 256 * 256;
    const size_t off_d = off_blo + (bytesB + 255) / 256 * 256;
    const size_t off_inst = off_d + (bytesD + 255) / 256 * 256;
    const size_t off_err = off_inst + 1024;
    if (cudaMalloc(&buf, off_err + 256) != cudaSuccess) return UBQP_ENOMEM;
    int rc = UBQP_OK;
    do {
        if (cudaMemset(buf, 0, off_err + 256) != cudaSuccess) { rc = UBQP_ECUDA; break; }
        std::vector<uint16_t> At((size_t)ld * ld, 0);   // A in the tiled layout of the solver
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) At[qbf_index((size_t)i, (size_t)j, (size_t)ld)] = A[i * n + j];
        if (cudaMemcpy(buf, At.data(), At.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy2D(buf + off_bhi, (size_t)ld * 2, Bhi, (size_t)n * 2, (size_t)n * 2, (size_t)R,
                         cudaMemcpyHostToDevice) != cudaSuccess ||
            (two && cudaMemcpy2D(buf + off_blo, (size_t)ld * 2, Blo, (size_t)n * 2, (size_t)n * 2, (size_t)R,
                                 cudaMemcpyHostToDevice) != cudaSuccess)) {
            rc = UBQP_ECUDA;
            break;
        }
        TcInst h;
        memset(&h, 0, sizeof(h));
        if (tc_encode_map(&h.tmA, buf, (int64_t)ld * ld / 64, 64, 128) != CUDA_SUCCESS ||
            tc_encode_map(&h.tmBhi, buf + off_bhi, rows_b, ld, bn) != CUDA_SUCCESS ||
            tc_encode_map(&h.tmBlo, buf + off_blo, rows_b, ld, bn) != CUDA_SUCCESS) {
            rc = UBQP_ECUDA;
            break;
        }
        h.n = (int)n;
        h.ld = ld;
        h.R = (int)R;
        h.lane0 = 0;
        h.m_tiles = ld / 128;
        h.n_tiles = n_tiles;
        h.bn = bn;
        h.two_terms = two ? 1 : 0;
        h.cluster0 = 0;
        if (cudaMemcpy(buf + off_inst, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) { rc = UBQP_ECUDA; break; }
        TcArgs a;
        memset(&a, 0, sizeof(a));
        a.inst = reinterpret_cast<const TcInst*>(buf + off_inst);
        a.ninst = 1;
        const bool persistent = cluster == -1;
        if (persistent && tcp_pick_stages(bn, two) < 2) { rc = UBQP_ENOTSUP; break; }
        a.stages = persistent ? tcp_pick_stages(bn, two) : tc_pick_stages(bn, two);
        a.tmem_cols = persistent ? tcp_tmem_cols(two) : tc_tmem_cols(bn, two);
        a.max_bn = bn;
        a.two_any = two ? 1 : 0;
        a.raw = reinterpret_cast<float*>(buf + off_d);
        a.err = reinterpret_cast<int32_t*>(buf + off_err);
        const int tiles = h.m_tiles * h.n_tiles;
        cudaError_t le;
        if (persistent) {
            le = tcp_launch(a, tiles, tcp_grid(a, tiles), nullptr);
        } else {
            const int S = cluster > 0 ? cluster : tc_pick_cluster(tiles, ld / 64, bn, two, a.stages, nsm);
            le = tc_launch(a, tiles, S, nullptr);
        }
        if (le != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            rc = UBQP_ECUDA;
            break;
        }
        int32_t err = 0;
        cudaMemcpy(&err, a.err, 4, cudaMemcpyDeviceToHost);
        if (err) { rc = UBQP_ETIMEOUT; break; }
        if (cudaMemcpy2D(D_out, (size_t)n * 4, a.raw, (size_t)ld * 4, (size_t)n * 4, (size_t)R,
                         cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = UBQP_ECUDA;
    } while (0);
    cudaFree(buf);
    return rc;
}
