// Row kernels shared by the two schedulers of phase A on CUDA cores (the lock-step tick
// kernel and the persistent lane loop): the dot products of matrix rows with the lane's
// input u held in shared memory, and the work of one (lane, row block) item.  Both
// schedulers call the same functions, so a lane's arithmetic does not depend on which one
// runs it.
#pragma once

#include "lane_update.cuh"

namespace ubqp {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// dot of one row with u (shared), FP32 row, 16-byte loads.  The four products of each
// 16-byte group are summed with FMAs and the group sum is added to a TwoSum-compensated
// accumulator: the error stays near 4 eps times the sum of |terms| instead of growing with
// the row length, at under 3 FP32 operations per matrix entry.
__device__ __forceinline__ void cacc4(float2& acc, float4 q, float4 u)
{
    float t = __fmul_rn(q.x, u.x);
    t = fmaf(q.y, u.y, t);
    t = fmaf(q.z, u.z, t);
    t = fmaf(q.w, u.w, t);
    float s, e;
    two_sum(acc.x, t, s, e);
    acc.x = s;
    acc.y += e;
}

__device__ __forceinline__ float4 ldg_stream(const float4* p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// dot of NR rows (1 or 2) with u: 16-byte groups at columns c, c + 32, c + 64, c + 96 (in
// float4 units) are loaded for every row before any is used, so each lane keeps 4 * NR
// loads in flight.  Group j goes to accumulator j & 1 of its row, in column order; the
// tails keep the same alternation, so the result does not depend on the unrolling or NR.
template <int NR>
__device__ __forceinline__ void rows_dot_f32(const float* const (&rows)[NR], const float* su, int ld, int lane,
                                             float (&out)[NR])
{
    const float4* u4 = reinterpret_cast<const float4*>(su);
    const int n4 = ld >> 2;
    float2 acc[NR][2];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = make_float2(0.f, 0.f);
    int c = lane;
    for (; c + 96 < n4; c += 128) {
        float4 q[NR][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < NR; ++r) q[r][j] = ldg_stream(reinterpret_cast<const float4*>(rows[r]) + c + 32 * j);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 u = u4[c + 32 * j];
#pragma unroll
            for (int r = 0; r < NR; ++r) cacc4(acc[r][j & 1], q[r][j], u);
        }
    }
    for (; c + 32 < n4; c += 64) {
        float4 q[NR][2];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < NR; ++r) q[r][j] = ldg_stream(reinterpret_cast<const float4*>(rows[r]) + c + 32 * j);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float4 u = u4[c + 32 * j];
#pragma unroll
            for (int r = 0; r < NR; ++r) cacc4(acc[r][j], q[r][j], u);
        }
    }
    for (; c < n4; c += 32) {
        const float4 u = u4[c];
#pragma unroll
        for (int r = 0; r < NR; ++r) cacc4(acc[r][0], ldg_stream(reinterpret_cast<const float4*>(rows[r]) + c), u);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const float2 a = csum_shfl_reduce(csum_merge(acc[r][0], acc[r][1]));
        out[r] = a.x + a.y;
    }
}

// dot of one row of the evaluation matrix (each FP64 entry q stored as FP32 hi + lo with
// hi + lo = q to about 2^-48) with a 0/1 vector: the products are the entries themselves,
// so TwoSum accumulation of hi and lo gives the FP64 row sum without FP64 arithmetic
// (exactly, for integer data).  Four 16-byte groups (eight entries) in flight per lane.
__device__ __forceinline__ double row_dot_eval(const float2* __restrict__ row, const float* su, int ld, int lane)
{
    const float4* r4 = reinterpret_cast<const float4*>(row);   // two entries per 16 bytes
    const float2* u2 = reinterpret_cast<const float2*>(su);
    const int n2 = ld >> 1;
    float2 ah = make_float2(0.f, 0.f), al = ah;
    int c = lane;
    for (; c + 96 < n2; c += 128) {
        float4 q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) q[j] = ldg_stream(r4 + c + 32 * j);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 u = u2[c + 32 * j];
            if (u.x != 0.f) { csum_add(ah, q[j].x); csum_add(al, q[j].y); }
            if (u.y != 0.f) { csum_add(ah, q[j].z); csum_add(al, q[j].w); }
        }
    }
    for (; c < n2; c += 32) {
        const float4 q = ldg_stream(r4 + c);
        const float2 u = u2[c];
        if (u.x != 0.f) { csum_add(ah, q.x); csum_add(al, q.y); }
        if (u.y != 0.f) { csum_add(ah, q.z); csum_add(al, q.w); }
    }
    ah = csum_shfl_reduce(ah);
    al = csum_shfl_reduce(al);
    return ((double)ah.x + (double)ah.y) + ((double)al.x + (double)al.y);
}

// u (written by the lane's last update, zero beyond n) into shared memory
__device__ __forceinline__ void item_load_u(const LaneDev& L, float* su)
{
    const float4* g4 = reinterpret_cast<const float4*>(L.vec + (size_t)V_U * L.ld);
    float4* s4 = reinterpret_cast<float4*>(su);
    for (int c = threadIdx.x; c < (L.ld >> 2); c += kThreads) s4[c] = g4[c];
}

// v_r = (row row0 + r of the phase's matrix) . u for r < rows, into sv[r]
__device__ __forceinline__ void item_rows(const LaneDev& L, int ph, int row0, int rows, const float* su, double* sv)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ld = L.ld;
    if (ph == PH_EVAL) {
        for (int r = warp; r < rows; r += kWarps) {
            double v = row_dot_eval(L.Qeval + (size_t)(row0 + r) * ld, su, ld, lane);
            if (lane == 0) sv[r] = v;
        }
    } else {
        // warp w takes rows w and w + kWarps together, then w + 2 kWarps, ...
        for (int r = warp; r < rows; r += 2 * kWarps) {
            const float* ra = L.Qoff + (size_t)(row0 + r) * ld;
            if (r + kWarps < rows) {
                const float* const rp[2] = {ra, ra + (size_t)kWarps * ld};
                float v[2];
                rows_dot_f32<2>(rp, su, ld, lane, v);
                if (lane == 0) {
                    sv[r] = (double)v[0];
                    sv[r + kWarps] = (double)v[1];
                }
            } else {
                const float* const rp[1] = {ra};
                float v[1];
                rows_dot_f32<1>(rp, su, ld, lane, v);
                if (lane == 0) sv[r] = (double)v[0];
            }
        }
    }
}

// per-row epilogue of the item's rows and its partial L.part[blk]; also counts the
// algorithmic bytes of the item when P.bytes is set: the stored entries of these rows once
// (FP32, or 8 bytes per entry of the evaluation matrix), the input vector once per lane
// (charged to block 0), and the per-row vectors the epilogue touches
__device__ __forceinline__ void item_finish(const LaneDev& L, int ph, int k, int blk, int row0, int rows,
                                            const double* sv, const Params& P)
{
    Acc a;
    a.zero();
    if ((int)threadIdx.x < rows) row_epilogue(L, ph, k, row0 + threadIdx.x, sv[threadIdx.x], a, P.tau_z);
    block_reduce_write<kWarps>(a, ph, L.part + blk, ph == PH_EVAL);
    if (P.bytes && threadIdx.x == 0) {
        unsigned long long by = (unsigned long long)rows * L.n * (ph == PH_EVAL ? 8ull : 4ull) +
                                (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
        atomicAdd(P.bytes, by);
    }
}

}  // namespace ubqp
