// Phase A on CUDA cores, lock-step scheduler: one launch per tick in which every active
// lane advances by one step.  v = Q_off u for each (lane, row block) item, then the per-row
// epilogue of the lane's phase (gradient of Alg. 2, eigen-solver matvec, Jacobi sweep,
// exact evaluation); the last CTA of a lane runs its update.  Persistent CTAs of 256
// threads pull items from a queue and stream rows from HBM into registers with 16-byte
// loads while u sits in shared memory.  The kernel is bound by the bytes of Q it reads:
// n * ld * 4 per lane per tick (FP32), 8 per entry for the evaluation tick.
//
// This file also holds the kernel that computes h and grad h for ubqp_penalized_eval
// (MODE_GRAD lanes), so the autograd path and the inner loop share one gradient kernel.
#include "gemv_rows.cuh"

namespace ubqp {

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
        const int row0 = it.y * A.rows_per_item;
        const int rows = min(A.rows_per_item, L.n - row0);
        if (s_ulane != it.x) item_load_u(L, su);   // consecutive items of one lane share u
        __syncthreads();
        if (threadIdx.x == 0) s_ulane = it.x;
        item_rows(L, ph, row0, rows, su, sv);
        __syncthreads();
        item_finish(L, ph, k, it.y, row0, rows, sv, A.P);
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

// persistent grid: every CTA that fits on the GPU at once, never more CTAs than items
int gemv_grid(int max_ld, int nitems)
{
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, phase_a_gemv_kernel, kThreads,
                                                                  (size_t)max_ld * sizeof(float));
    if (e != cudaSuccess || per < 1) {
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
