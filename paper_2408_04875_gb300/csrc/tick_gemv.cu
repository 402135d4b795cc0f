// Phase A on CUDA cores: v = Q_off u for one row block of one lane, then the per-row
// epilogue of the lane's phase (gradient of Alg. 2, eigen-solver matvec, Jacobi sweep,
// exact evaluation).  One CTA of 256 threads per (lane, row block); each warp streams
// whole rows with 16-byte loads while u sits in shared memory.  The kernel is bound by
// the bytes of Q it reads: n * ld * 4 per lane per tick (FP32), 8 per entry for the
// evaluation tick that reads the original FP64 matrix.
//
// The same kernel computes h and grad h for ubqp_penalized_eval (MODE_GRAD lanes), so
// the autograd path and the inner loop share one gradient kernel.
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
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// two rows at once (independent load streams), same arithmetic as row_dot_f32
__device__ __forceinline__ void row_dot2_f32(const float* __restrict__ ra, const float* __restrict__ rb,
                                             const float* su, int ld, int lane, float& va, float& vb)
{
    const float4* a4 = reinterpret_cast<const float4*>(ra);
    const float4* b4 = reinterpret_cast<const float4*>(rb);
    const float4* u4 = reinterpret_cast<const float4*>(su);
    const int n4 = ld >> 2;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
    int c = lane;
    for (; c + 32 < n4; c += 64) {
        const float4 qa0 = ldg_stream(a4 + c), qa1 = ldg_stream(a4 + c + 32);
        const float4 qb0 = ldg_stream(b4 + c), qb1 = ldg_stream(b4 + c + 32);
        const float4 u0 = u4[c], u1 = u4[c + 32];
        cacc4(a0, qa0, u0);
        cacc4(b0, qb0, u0);
        cacc4(a1, qa1, u1);
        cacc4(b1, qb1, u1);
    }
    for (; c < n4; c += 32) {
        const float4 u0 = u4[c];
        cacc4(a0, ldg_stream(a4 + c), u0);
        cacc4(b0, ldg_stream(b4 + c), u0);
    }
    float2 a = csum_shfl_reduce(csum_merge(a0, a1));
    float2 b = csum_shfl_reduce(csum_merge(b0, b1));
    va = a.x + a.y;
    vb = b.x + b.y;
}

__device__ __forceinline__ float row_dot_f32(const float* __restrict__ row, const float* su, int ld,
                                             int lane)
{
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const float4* u4 = reinterpret_cast<const float4*>(su);
    const int n4 = ld >> 2;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int c = lane;
    for (; c + 96 < n4; c += 128) {
        float4 q0 = __ldg(r4 + c), q1 = __ldg(r4 + c + 32), q2 = __ldg(r4 + c + 64), q3 = __ldg(r4 + c + 96);
        cacc4(a0, q0, u4[c]);
        cacc4(a1, q1, u4[c + 32]);
        cacc4(a2, q2, u4[c + 64]);
        cacc4(a3, q3, u4[c + 96]);
    }
    for (; c < n4; c += 32) cacc4(a0, __ldg(r4 + c), u4[c]);
    float2 a = csum_merge(csum_merge(a0, a1), csum_merge(a2, a3));
    a = csum_shfl_reduce(a);
    return a.x + a.y;
}

// dot of one row of the evaluation matrix (each FP64 entry q stored as FP32 hi + lo with
// hi + lo = q to about 2^-48) with a 0/1 vector: the products are the entries themselves,
// so TwoSum accumulation of hi and lo gives the FP64 row sum without FP64 arithmetic
// (exactly, for integer data)
__device__ __forceinline__ double row_dot_eval(const float2* __restrict__ row, const float* su, int ld,
                                               int lane)
{
    const float4* r4 = reinterpret_cast<const float4*>(row);   // two entries per 16 bytes
    const float2* u2 = reinterpret_cast<const float2*>(su);
    const int n2 = ld >> 1;
    float2 ah = make_float2(0.f, 0.f), al = ah;
    for (int c = lane; c < n2; c += 32) {
        float4 q = __ldg(r4 + c);
        float2 u = u2[c];
        if (u.x != 0.f) { csum_add(ah, q.x); csum_add(al, q.y); }
        if (u.y != 0.f) { csum_add(ah, q.z); csum_add(al, q.w); }
    }
    ah = csum_shfl_reduce(ah);
    al = csum_shfl_reduce(al);
    return ((double)ah.x + (double)ah.y) + ((double)al.x + (double)al.y);
}

// generic (unaligned, unpadded) row dot for user matrices of penalized_eval
template <typename T>
__device__ __forceinline__ T row_dot_plain(const T* __restrict__ row, const T* su, int n, int lane)
{
    T a0 = 0, a1 = 0;
    int c = lane;
    for (; c + 32 < n; c += 64) {
        a0 += row[c] * su[c];
        a1 += row[c + 32] * su[c + 32];
    }
    for (; c < n; c += 32) a0 += row[c] * su[c];
    T a = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// ---------------------------------------------------------------------------------
// solver lanes (FP32 GEMV path)
__global__ void __launch_bounds__(kThreads, 4) phase_a_gemv_kernel(TickArgs A)
{
    // Persistent: CTAs pull (lane, row-block) items from a queue until it is empty; the
    // items of the largest lanes come first.  u stays in shared memory while consecutive
    // items belong to the same lane.
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* su = reinterpret_cast<float*>(smem_raw);
    __shared__ double sv[kThreads];
    __shared__ int s_item, s_ulane, is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_ulane = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= A.nitems) break;
        const int2 it = A.items[item];
        const LaneDev& L = A.lanes[it.x];
        const int ph = L.st->phase;
        if (ph == PH_DONE || ph == PH_GRAD) {
            __syncthreads();
            continue;
        }
        const int k = L.st->k;
        const int ld = L.ld;
        const int row0 = it.y * A.rows_per_item;
        const int rows = min(A.rows_per_item, L.n - row0);

        // u (written by the update of the previous tick, zero beyond n)
        if (s_ulane != it.x) {
            const float4* g4 = reinterpret_cast<const float4*>(L.vec + (size_t)V_U * ld);
            float4* s4 = reinterpret_cast<float4*>(su);
            for (int c = threadIdx.x; c < (ld >> 2); c += kThreads) s4[c] = g4[c];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_ulane = it.x;

        if (ph == PH_EVAL) {
            for (int r = warp; r < rows; r += kWarps) {
                double v = row_dot_eval(L.Qeval + (size_t)(row0 + r) * ld, su, ld, lane);
                if (lane == 0) sv[r] = v;
            }
        } else {
            for (int r = warp; r < rows; r += 2 * kWarps) {
                const int r2 = r + kWarps < rows ? r + kWarps : r;
                float va, vb;
                row_dot2_f32(L.Qoff + (size_t)(row0 + r) * ld, L.Qoff + (size_t)(row0 + r2) * ld, su, ld, lane,
                             va, vb);
                if (lane == 0) {
                    sv[r] = (double)va;
                    sv[r2] = (double)vb;
                }
            }
        }
        __syncthreads();

        Acc a;
        a.zero();
        if ((int)threadIdx.x < rows) row_epilogue(L, ph, k, row0 + threadIdx.x, sv[threadIdx.x], a, A.P.tau_z);
        block_reduce_write<kWarps>(a, ph, L.part + it.y, ph == PH_EVAL);
        if (A.P.bytes && threadIdx.x == 0) {
            // stored entries of these rows once (FP32, or the 8-byte evaluation matrix), the
            // input vector once per lane, and the per-row vectors the epilogue touches
            unsigned long long by = (unsigned long long)rows * L.n * (ph == PH_EVAL ? 8ull : 4ull) +
                                    (it.y == 0 ? 4ull * L.n : 0ull) + 16ull * rows;
            atomicAdd(A.P.bytes, by);
        }
        if (A.fused) {
            // every CTA publishes its partial and epilogue writes, then counts itself in; the
            // CTA that completes the lane's count runs the lane's update.  No CTA waits.
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) is_last = (atomicAdd(L.counter, 1u) == (unsigned)(L.nblk - 1));
            __syncthreads();
            if (is_last) {
                __threadfence();
                lane_update(L, A.P, A.active_count);
                if (threadIdx.x == 0) {
                    *L.counter = 0u;
                    s_ulane = -1;
                }
            }
        }
        __syncthreads();
    }
    // the last CTA to leave resets the queue for the next tick
    if (threadIdx.x == 0 && atomicAdd(A.done, 1) == (int)gridDim.x - 1) {
        *A.work = 0;
        *A.done = 0;
    }
}

// ---------------------------------------------------------------------------------
// gradient lanes: h and g of problem (p) for one point, matrix of type T
template <typename T>
__global__ void __launch_bounds__(kThreads) phase_a_grad_kernel(TickArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    __shared__ T sv[kThreads];

    const int2 it = A.items[blockIdx.x];
    const LaneDev& L = A.lanes[it.x];
    const int n = L.n;
    const int row0 = it.y * A.rows_per_item;
    const int rows = min(A.rows_per_item, n - row0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T* Q = static_cast<const T*>(L.gQ);
    const T* x = static_cast<const T*>(L.gx);
    const T* b = static_cast<const T*>(L.gb);
    const T* p = static_cast<const T*>(L.gp);
    T* g = static_cast<T*>(L.gg);

    for (int c = threadIdx.x; c < n; c += kThreads) su[c] = x[c];
    __syncthreads();
    for (int r = warp; r < rows; r += kWarps) {
        T v = row_dot_plain<T>(Q + (size_t)(row0 + r) * L.gld, su, n, lane);
        if (lane == 0) sv[r] = v;
    }
    __syncthreads();

    // g = 2 (Q - Diag p) x + b + p;  h contribution x_i (Qx)_i + b_i x_i + p_i (x_i - x_i^2)
    double hpart = 0.0;
    if ((int)threadIdx.x < rows) {
        const int i = row0 + threadIdx.x;
        T v = sv[threadIdx.x];
        T xi = su[i];
        T bi = b ? b[i] : T(0);
        T pi = p ? p[i] : T(0);
        if (g) g[i] = T(2) * v - T(2) * pi * xi + bi + pi;
        hpart = (double)(xi * (v + bi + pi - pi * xi));
    }
    hpart = dsum_shfl_reduce(hpart);
    __shared__ double sh[kWarps];
    if (lane == 0) sh[warp] = hpart;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sh[w];
        L.part[it.y].f = t;
    }
}

template <typename T>
__global__ void grad_reduce_kernel(const LaneDev* lanes, int nlanes, T* h_out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlanes) return;
    const LaneDev& L = lanes[l];
    double t = 0.0;
    for (int b = 0; b < L.nblk; ++b) t += L.part[b].f;
    h_out[l] = (T)t;
}

cudaError_t prepare_phase_a_gemv(int max_ld)
{
    size_t smem = (size_t)max_ld * sizeof(float);
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(phase_a_gemv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int gemv_grid(int max_ld, int nitems)
{
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, phase_a_gemv_kernel, kThreads,
                                                      (size_t)max_ld * sizeof(float)) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    int g = sms * per;
    return nitems < g ? nitems : g;
}

cudaError_t launch_phase_a_gemv_f32(const TickArgs& a, cudaStream_t s)
{
    // shared: u of the widest lane (ld floats); rows_per_item <= kThreads
    size_t smem = (size_t)a.max_ld * sizeof(float);
    phase_a_gemv_kernel<<<a.grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_phase_a_grad(const TickArgs& a, int dtype, int64_t n, cudaStream_t s)
{
    size_t smem = (size_t)n * (dtype == 1 ? sizeof(double) : sizeof(float));
    if (dtype == 1) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(phase_a_grad_kernel<double>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        phase_a_grad_kernel<double><<<a.nitems, kThreads, smem, s>>>(a);
    } else {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(phase_a_grad_kernel<float>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        phase_a_grad_kernel<float><<<a.nitems, kThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const LaneDev* lanes, int nlanes, void* h_out, int dtype, cudaStream_t s)
{
    int threads = 128, blocks = (nlanes + threads - 1) / threads;
    if (dtype == 1) grad_reduce_kernel<double><<<blocks, threads, 0, s>>>(lanes, nlanes, (double*)h_out);
    else grad_reduce_kernel<float><<<blocks, threads, 0, s>>>(lanes, nlanes, (float*)h_out);
    return cudaGetLastError();
}

}  // namespace ubqp
