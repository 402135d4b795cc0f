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

// FP64 rows (the penalized objective in FP64 only): the two products of a 16-byte group
// summed with an FMA, then added to a plain FP64 accumulator (each lane sums about n / 64
// groups, so the accumulated rounding stays near 1e-14 of the sum of |terms|)
__device__ __forceinline__ void cacc4(double& acc, double2 q, double2 u) { acc += fma(q.y, u.y, q.x * u.x); }

__device__ __forceinline__ double2 ldg_stream(const double2* p)
{
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

// element type -> its 16-byte group, the accumulator of a row dot, and the warp reduction
template <typename T> struct RowT;
template <> struct RowT<float> {
    using V = float4;
    using A = float2;   // TwoSum-compensated (sum, error)
    static constexpr int W = 4;
    __device__ static A zero() { return make_float2(0.f, 0.f); }
    __device__ static void add1(A& a, float q, float u) { csum_add(a, __fmul_rn(q, u)); }
    __device__ static float finish(A a0, A a1)
    {
        const float2 a = csum_shfl_reduce(csum_merge(a0, a1));
        return a.x + a.y;
    }
    __device__ static V lds(const float* s, int e) { return make_float4(s[e], s[e + 1], s[e + 2], s[e + 3]); }
};
template <> struct RowT<double> {
    using V = double2;
    using A = double;
    static constexpr int W = 2;
    __device__ static A zero() { return 0.0; }
    __device__ static void add1(A& a, double q, double u) { a = fma(q, u, a); }
    __device__ static double finish(A a0, A a1) { return dsum_shfl_reduce(a0 + a1); }
    __device__ static V lds(const double* s, int e) { return make_double2(s[e], s[e + 1]); }
};

// dot of NR rows (1 or 2) with u: 16-byte groups at columns c, c + 32, c + 64, c + 96 (in
// group units) are loaded for every row before any is used, so each lane keeps 4 * NR
// loads in flight.  Group j goes to accumulator j & 1 of its row, in column order; the
// tails keep the same alternation, so the result does not depend on the unrolling or NR.
// The rows start 16-byte aligned and hold ngrp whole groups (the solver's padded rows:
// ngrp = ld / 4, so every column is covered); u is read in groups from shared memory, at
// element offset uoff.  UAL: uoff is a multiple of the group width (16-byte loads of u).
template <typename T, int NR, bool UAL>
__device__ __forceinline__ void rows_dot_body(const T* const (&rows)[NR], const T* su, int uoff, int ngrp, int lane,
                                              typename RowT<T>::A (&acc)[NR][2])
{
    using R = RowT<T>;
    using V = typename R::V;
    constexpr int W = R::W;
    auto ul = [&](int g) -> V {
        if constexpr (UAL) return reinterpret_cast<const V*>(su + uoff)[g];
        else return R::lds(su, uoff + W * g);
    };
    int c = lane;
    for (; c + 96 < ngrp; c += 128) {
        V q[NR][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < NR; ++r) q[r][j] = ldg_stream(reinterpret_cast<const V*>(rows[r]) + c + 32 * j);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const V u = ul(c + 32 * j);
#pragma unroll
            for (int r = 0; r < NR; ++r) cacc4(acc[r][j & 1], q[r][j], u);
        }
    }
    for (; c + 32 < ngrp; c += 64) {
        V q[NR][2];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < NR; ++r) q[r][j] = ldg_stream(reinterpret_cast<const V*>(rows[r]) + c + 32 * j);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const V u = ul(c + 32 * j);
#pragma unroll
            for (int r = 0; r < NR; ++r) cacc4(acc[r][j], q[r][j], u);
        }
    }
    for (; c < ngrp; c += 32) {
        const V u = ul(c);
#pragma unroll
        for (int r = 0; r < NR; ++r) cacc4(acc[r][0], ldg_stream(reinterpret_cast<const V*>(rows[r]) + c), u);
    }
}

// the solver's rows: 16-byte aligned, ld (a multiple of 4) columns, zero beyond n
template <int NR>
__device__ __forceinline__ void rows_dot_f32(const float* const (&rows)[NR], const float* su, int ld, int lane,
                                             float (&out)[NR])
{
    float2 acc[NR][2];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = make_float2(0.f, 0.f);
    rows_dot_body<float, NR, true>(rows, su, 0, ld >> 2, lane, acc);
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] = RowT<float>::finish(acc[r][0], acc[r][1]);
}

// a caller's rows of n entries (row-major, no padding; the two rows of a pair lie 8 rows
// apart, so they share their alignment).  The first `head` entries before the first 16-byte
// boundary and the `tail` entries after the last whole group are taken one by one by the
// first lanes; the groups in between run the solver's loop above.
template <typename T, int NR>
__device__ __forceinline__ void rows_dot_any(const T* const (&rows)[NR], const T* su, int n, int lane,
                                             T (&out)[NR])
{
    using R = RowT<T>;
    constexpr int W = R::W;
    const int mis = (int)((reinterpret_cast<uintptr_t>(rows[0]) & 15u) / sizeof(T));
    const int head = min((W - mis) % W, n);
    const int ngrp = (n - head) / W;
    const int tail = n - head - W * ngrp;
    typename R::A acc[NR][2];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = R::zero();
    const T* body[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) body[r] = rows[r] + head;
    if (head % W == 0) rows_dot_body<T, NR, true>(body, su, head, ngrp, lane, acc);
    else rows_dot_body<T, NR, false>(body, su, head, ngrp, lane, acc);
    if (lane < head) {
#pragma unroll
        for (int r = 0; r < NR; ++r) R::add1(acc[r][1], rows[r][lane], su[lane]);
    }
    if (lane < tail) {
        const int e = head + W * ngrp + lane;
#pragma unroll
        for (int r = 0; r < NR; ++r) R::add1(acc[r][1], rows[r][e], su[e]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] = R::finish(acc[r][0], acc[r][1]);
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

// u (written by the lane's last update, zero beyond n) into shared memory; for a gradient
// lane (penalized objective) the caller's point x, of the caller's element type T
template <typename T = float>
__device__ __forceinline__ void item_load_u(const LaneDev& L, T* su)
{
    if (L.mode == MODE_GRAD) {
        const T* x = static_cast<const T*>(L.gx);
        for (int c = threadIdx.x; c < L.n; c += kThreads) su[c] = x[c];
        return;
    }
    if constexpr (sizeof(T) == sizeof(float)) {
        const float4* g4 = reinterpret_cast<const float4*>(L.vec + (size_t)V_U * L.ld);
        float4* s4 = reinterpret_cast<float4*>(su);
        for (int c = threadIdx.x; c < (L.ld >> 2); c += kThreads) s4[c] = g4[c];
    }
}

// Q'_off rows from the sliced storage: an item of 32 * m rows (m = 1, 2, 4 or 8 slices) with
// L.spwps = 8 / m warps per slice; the warps of a slice take consecutive shares of its stored
// entries (lane r: row r of the slice), groups of four products summed with FMAs and added to
// a TwoSum-compensated sum, and the shares are merged per row in share order.
__device__ __forceinline__ void item_rows_sell(const LaneDev& L, int row0, int rows, const float* su, double* sv,
                                               int lane, int warp)
{
    __shared__ float2 s_share[kThreads];
    const int wps = L.spwps;
    const int sl = warp / wps, part = warp - sl * wps;
    float2 acc = make_float2(0.f, 0.f);
    if (sl * 32 < rows) {
        const int64_t b = L.spo[(row0 >> 5) + sl];
        const int width = (int)((L.spo[(row0 >> 5) + sl + 1] - b) >> 5);
        const int k0 = width * part / wps, k1 = width * (part + 1) / wps;
        const float* V = L.spv + b + lane;
        const uint16_t* C = L.spc + b + lane;
        int k = k0;
        for (; k + 8 <= k1; k += 8) {
            float q[8];
            int c[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                q[j] = __ldg(V + 32 * (k + j));
                c[j] = __ldg(C + 32 * (k + j));
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float t = __fmul_rn(q[4 * h], su[c[4 * h]]);
                t = fmaf(q[4 * h + 1], su[c[4 * h + 1]], t);
                t = fmaf(q[4 * h + 2], su[c[4 * h + 2]], t);
                t = fmaf(q[4 * h + 3], su[c[4 * h + 3]], t);
                csum_add(acc, t);
            }
        }
        for (; k < k1; ++k) csum_add(acc, __fmul_rn(__ldg(V + 32 * k), su[__ldg(C + 32 * k)]));
    }
    s_share[(sl * 32 + lane) * wps + part] = acc;
    __syncthreads();
    if ((int)threadIdx.x < rows) {
        float2 a = s_share[threadIdx.x * wps];
        for (int q = 1; q < wps; ++q) a = csum_merge(a, s_share[threadIdx.x * wps + q]);
        sv[threadIdx.x] = (double)(a.x + a.y);
    }
}

// the solver's matrices: the FP32 hi/lo evaluation rows (PH_EVAL), the sliced storage or the
// padded Q'_off rows
__device__ __forceinline__ void item_rows_solver(const LaneDev& L, int ph, int row0, int rows, const float* su,
                                                 double* sv, int lane, int warp)
{
    const int ld = L.ld;
    if (ph != PH_EVAL && L.spv) {
        item_rows_sell(L, row0, rows, su, sv, lane, warp);
        return;
    }
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


// v_r = (row row0 + r of the phase's matrix) . u for r < rows, into sv[r]
template <typename T = float>
__device__ __forceinline__ void item_rows(const LaneDev& L, int ph, int row0, int rows, const T* su, double* sv)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (ph == PH_GRAD) {
        // the caller's Q (n x n, row stride gld, element type T), diagonal included
        const T* Q = static_cast<const T*>(L.gQ);
        for (int r = warp; r < rows; r += 2 * kWarps) {
            const T* ra = Q + (size_t)(row0 + r) * L.gld;
            if (r + kWarps < rows) {
                const T* const rp[2] = {ra, ra + (size_t)kWarps * L.gld};
                T v[2];
                rows_dot_any<T, 2>(rp, su, L.n, lane, v);
                if (lane == 0) {
                    sv[r] = (double)v[0];
                    sv[r + kWarps] = (double)v[1];
                }
            } else {
                const T* const rp[1] = {ra};
                T v[1];
                rows_dot_any<T, 1>(rp, su, L.n, lane, v);
                if (lane == 0) sv[r] = (double)v[0];
            }
        }
        return;
    }
    if constexpr (sizeof(T) == sizeof(float)) item_rows_solver(L, ph, row0, rows, su, sv, lane, warp);
}

// Gradient lanes (the penalized objective of Sec. 4.1, problem (p)): row i received
// v = (Q x)_i of the caller's Q (diagonal included); the epilogue writes
//     g_i = 2 v - 2 p_i x_i + b_i + p_i          (grad of h = x^T (Q - P*) x + (b + p)^T x)
// and adds h_i = x_i (v + b_i + p_i - p_i x_i) to the item's FP64 partial sum of h.
template <typename T>
__device__ __forceinline__ void item_finish_grad(const LaneDev& L, int blk, int row0, int rows, const double* sv,
                                                 const T* su)
{
    Acc a;
    a.zero();
    if ((int)threadIdx.x < rows) {
        const int i = row0 + threadIdx.x;
        const T v = (T)sv[threadIdx.x];
        const T x = su[i];
        const T b = L.gb ? static_cast<const T*>(L.gb)[i] : T(0);
        const T p = L.gp ? static_cast<const T*>(L.gp)[i] : T(0);
        if (L.gg) static_cast<T*>(L.gg)[i] = T(2) * v - T(2) * p * x + b + p;
        a.f = (double)x * ((double)v + (double)b + (double)p - (double)p * (double)x);
    }
    block_reduce_write<kWarps>(a, PH_GRAD, L.part + blk, true);
}

// per-row epilogue of the item's rows and its partial L.part[blk]; also counts the
// algorithmic bytes of the item when P.bytes is set: the stored entries of these rows once
// (FP32, or 8 bytes per entry of the evaluation matrix), the input vector once per lane
// (charged to block 0), and the per-row vectors the epilogue touches
// (sym_parts > 0: the rows' products came from the symmetric tiles, and the item read
// sym_parts partial values per row instead of matrix rows)
__device__ __forceinline__ void item_finish(const LaneDev& L, int ph, int k, int blk, int row0, int rows,
                                            const double* sv, const Params& P, int sym_parts = 0)
{
    Acc a;
    a.zero();
    if ((int)threadIdx.x < rows) row_epilogue(L, ph, k, row0 + threadIdx.x, sv[threadIdx.x], a, P.tau_z);
    block_reduce_write<kWarps>(a, ph, L.part + blk, ph == PH_EVAL);
    if (P.bytes && threadIdx.x == 0) {
        unsigned long long by = sym_parts > 0
                                    ? (unsigned long long)rows * (unsigned long long)sym_parts * 4ull + 16ull * rows
                                    : (unsigned long long)rows * L.n * (ph == PH_EVAL ? 8ull : 4ull) +
                                          (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
        if (L.spv && ph != PH_EVAL)   // the item's stored entries (4-byte value, 2-byte column)
            by = 6ull * (unsigned long long)(L.spo[(row0 + rows + 31) >> 5] - L.spo[row0 >> 5]) +
                 (blk == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
        atomicAdd(P.bytes, by);
    }
}

// ---------------------------------------------------------------------------------
// Symmetric storage (persistent lane loop).  Q_off is symmetric, so only its upper
// triangle is stored, as kSymT x kSymT FP32 tiles (I <= J, row-major inside a tile) packed
// row by row: tile t of the sequence (0,0), (0,1), .., (0,nb-1), (1,1), ...  One read of a
// tile gives two products: its rows times u_J (for the rows of block I) and its columns
// times u_I (for the rows of block J); a diagonal tile is stored whole and gives its row
// products only.  Each product is a partial vector of kSymT values, written to
// pbuf[K * ld + row] with K the other block index, so that a row of block b finds its nb
// partials at pbuf[K * ld + row], K = 0 .. nb-1, from the tiles (b, K) or (K, b).  A second
// stage sums them in that order for each row block and runs the usual epilogue.
// tile t -> (I, J), I <= J, in the row-by-row packing of an nb x nb upper triangle
__device__ __forceinline__ void sym_tile_ij(int t, int nb, int& I, int& J)
{
    // first tile of row i: f(i) = i nb - i (i - 1) / 2; take the largest i with f(i) <= t
    const float b2 = 2.f * nb + 1.f;
    int i = (int)floorf((b2 - sqrtf(fmaxf(b2 * b2 - 8.f * (float)t, 0.f))) * 0.5f);
    i = max(0, min(i, nb - 1));
    while (i > 0 && i * nb - i * (i - 1) / 2 > t) --i;
    while (i + 1 < nb && (i + 1) * nb - (i + 1) * i / 2 <= t) ++i;
    I = i;
    J = i + (t - (i * nb - i * (i - 1) / 2));
}

// one tile of one lane: the row products go to pbuf[J][rows of I] and the column products of
// this thread's warp to s_colw (8 warps x kSymT, merged by the caller).  Warp w takes tile
// rows 16 w .. 16 w + 15 in two passes of 8, lane l columns 4 l .. 4 l + 3.  Row products: the
// four products of a lane summed with FMAs, then the 8 rows of a pass reduced over the 32
// lanes by a butterfly that halves the values each lane holds at every stage (9 shuffles for
// 8 rows; afterwards lane l holds row (l >> 2) & 7).  Column products: FMAs over the warp's
// 16 rows.  u_J (this lane's four columns) and u_I (each pass's rows) are read straight from
// the lane's input vector with the tile's loads.
// (Measured on the 40-lane sweep: 128 x 128 tiles 18.98 s per step; 256 x 256 tiles 21.8 s,
// too few work items once the small lanes are one tile each.)
__device__ __forceinline__ void sym_tile_part(const SymLane& S, const LaneDev& L, int t, float (*s_colw)[kSymT],
                                              const Params& P)
{
    static_assert(kSymT == 128 && kThreads == 256, "the mapping below is written for 128 x 128 tiles");
    int I, J;
    sym_tile_ij(t, S.nb, I, J);
    const int ld = L.ld;
    const float* u = L.vec + (size_t)V_U * ld;
    const float4 uj = reinterpret_cast<const float4*>(u + J * kSymT)[threadIdx.x & 31];
    const float4* tile = reinterpret_cast<const float4*>(S.Qsym + (size_t)t * kSymT * kSymT);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
    float* rowdst = S.pbuf + (size_t)J * ld + I * kSymT;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r0 = warp * 16 + h * 8;
        float4 q[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) q[r] = ldg_stream(tile + (size_t)(r0 + r) * (kSymT / 4) + lane);
        const float4 ui0 = reinterpret_cast<const float4*>(u + I * kSymT + r0)[0];
        const float4 ui1 = reinterpret_cast<const float4*>(u + I * kSymT + r0)[1];
        const float uis[8] = {ui0.x, ui0.y, ui0.z, ui0.w, ui1.x, ui1.y, ui1.z, ui1.w};
        float v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float a = __fmul_rn(q[r].x, uj.x);
            a = fmaf(q[r].y, uj.y, a);
            a = fmaf(q[r].z, uj.z, a);
            v[r] = fmaf(q[r].w, uj.w, a);
            const float ui = uis[r];
            c0 = fmaf(q[r].x, ui, c0);
            c1 = fmaf(q[r].y, ui, c1);
            c2 = fmaf(q[r].z, ui, c2);
            c3 = fmaf(q[r].w, ui, c3);
        }
        // butterfly: lanes with the stage's bit set keep the upper half of their rows
        {
            const bool up = lane & 16;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float keep = up ? v[j + 4] : v[j], send = up ? v[j] : v[j + 4];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
        }
        {
            const bool up = lane & 8;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float keep = up ? v[j + 2] : v[j], send = up ? v[j] : v[j + 2];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
        }
        {
            const bool up = lane & 4;
            const float keep = up ? v[1] : v[0], send = up ? v[0] : v[1];
            v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
        if ((lane & 3) == 0) rowdst[r0 + ((lane >> 2) & 7)] = v[0];
    }
    s_colw[warp][4 * lane + 0] = c0;
    s_colw[warp][4 * lane + 1] = c1;
    s_colw[warp][4 * lane + 2] = c2;
    s_colw[warp][4 * lane + 3] = c3;
    if (P.bytes && threadIdx.x == 0) {
        // the tile's entries inside the matrix once, u_I and u_J, the partial vectors written
        const unsigned long long ri = (unsigned long long)min(kSymT, L.n - I * kSymT);
        const unsigned long long cj = (unsigned long long)min(kSymT, L.n - J * kSymT);
        atomicAdd(P.bytes, ri * cj * 4ull + 2ull * kSymT * 4ull + (I != J ? 2ull : 1ull) * kSymT * 4ull);
    }
}

// one ring entry of the first stage: tiles kSymGroup g .. kSymGroup g + kSymGroup - 1 of a lane
// (fewer at the end).  The column products of every tile off the diagonal are merged over the
// 8 warps in order with TwoSum, after one barrier, by one 128-thread half of the CTA per tile.
__device__ __forceinline__ void sym_group_item(const SymLane& S, const LaneDev& L, int g,
                                               float (*s_col)[kWarps][kSymT], const Params& P)
{
    static_assert(kSymGroup * kSymT == kThreads, "one half of the CTA merges each tile's columns");
    const int t0 = g * kSymGroup;
#pragma unroll 1
    for (int k = 0; k < kSymGroup && t0 + k < S.ntiles; ++k) sym_tile_part(S, L, t0 + k, s_col[k], P);
    __syncthreads();
    const int k = threadIdx.x / kSymT, c = threadIdx.x % kSymT;
    if (t0 + k < S.ntiles) {
        int I, J;
        sym_tile_ij(t0 + k, S.nb, I, J);
        if (I != J) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) csum_add(acc, s_col[k][w][c]);
            S.pbuf[(size_t)I * L.ld + J * kSymT + c] = acc.x + acc.y;
        }
    }
}

// row products of block b from its nb partial vectors, summed in K order with TwoSum
__device__ __forceinline__ void sym_block_sums(const SymLane& S, const LaneDev& L, int b, int rows, double* sv)
{
    if ((int)threadIdx.x < rows) {
        const float* p = S.pbuf + b * kSymT + threadIdx.x;
        float2 acc = make_float2(0.f, 0.f);
        for (int K = 0; K < S.nb; ++K) csum_add(acc, p[(size_t)K * L.ld]);
        sv[threadIdx.x] = (double)(acc.x + acc.y);
    }
}

}  // namespace ubqp
