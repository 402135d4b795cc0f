// Phase A on CUDA cores, lock-step scheduler: one launch per tick in which every active
// lane advances by one step.  v = Q_off u for each (lane, row block) item, then the per-row
// epilogue of the lane's phase (gradient of Alg. 2, eigen-solver matvec, Jacobi sweep,
// exact evaluation); the last CTA of a lane runs its update.  Persistent CTAs of 256
// threads pull items from a queue and stream rows from HBM into registers with 16-byte
// loads while u sits in shared memory.  The kernel is bound by the bytes of Q it reads:
// n * ld * 4 per lane per tick (FP32), 8 per entry for the evaluation tick.
//
// The same kernel computes h and grad h of problem (p) for ubqp_penalized_eval: those
// lanes (MODE_GRAD) read the caller's Q rows with the inner loop's row dot (gemv_rows.cuh)
// and finish with the gradient epilogue; the FP32 instance is the one the inner loop runs,
// the FP64 instance the same source on FP64 data.
#include "gemv_rows.cuh"

namespace ubqp {

// ---------------------------------------------------------------------------------
// solver lanes (FP32) and gradient lanes (FP32 or FP64, element type T)
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) phase_a_gemv_kernel(TickArgs A)
{
    // Persistent: CTAs pull (lane, row-block) items from a queue until it is empty; the
    // items of the largest lanes come first.  u stays in shared memory while consecutive
    // items belong to the same lane.
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
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
        const bool grad = L.mode == MODE_GRAD;
        const int ph = grad ? (int)PH_GRAD : L.st->phase;
        if (ph == PH_DONE) {
            __syncthreads();
            continue;
        }
        const int k = grad ? 0 : L.st->k;
        const int row0 = it.y * A.rows_per_item;
        const int rows = min(A.rows_per_item, L.n - row0);
        if (s_ulane != it.x) item_load_u(L, su);   // consecutive items of one lane share u
        __syncthreads();
        if (threadIdx.x == 0) s_ulane = it.x;
        item_rows<T>(L, ph, row0, rows, su, sv);
        __syncthreads();
        if (grad) item_finish_grad<T>(L, it.y, row0, rows, sv, su);
        else item_finish(L, ph, k, it.y, row0, rows, sv, A.P);
        if (A.fused && !grad) {
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

// descriptors and work items of `batch` gradient lanes and the cleared queue counters, written
// on the device (no host staging): point r has blocks (r, 0 .. nblk-1)
__global__ void grad_setup_kernel(LaneDev* lanes, int2* items, int32_t* queue, Partial* part, const void* Q,
                                  const void* b, const void* p, const void* x, void* g, int n, int batch, int nblk,
                                  int es)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid < 2) queue[tid] = 0;
    if (tid < batch) {
        LaneDev L;
        memset(&L, 0, sizeof(L));
        L.n = n;
        L.ld = n;
        L.mode = MODE_GRAD;
        L.nblk = nblk;
        L.part = part + (size_t)tid * nblk;
        L.gQ = Q;
        L.gb = b;
        L.gp = p;
        L.gx = static_cast<const char*>(x) + (size_t)tid * n * es;
        L.gg = g ? static_cast<char*>(g) + (size_t)tid * n * es : nullptr;
        L.gld = n;
        lanes[tid] = L;
    }
    for (int t = tid; t < batch * nblk; t += gridDim.x * blockDim.x) items[t] = make_int2(t / nblk, t % nblk);
}

cudaError_t launch_grad_setup(LaneDev* lanes, int2* items, int32_t* queue, Partial* part, const void* Q, const void* b,
                              const void* p, const void* x, void* g, int n, int batch, int nblk, int es, cudaStream_t s)
{
    const int work = batch * nblk > batch ? batch * nblk : batch;
    grad_setup_kernel<<<(work + 255) / 256, 256, 0, s>>>(lanes, items, queue, part, Q, b, p, x, g, n, batch, nblk, es);
    return cudaGetLastError();
}

// vector-Jacobian product of h (backward of the penalized objective) for `batch` points:
//   gx[r][i] = go[r] g[r][i],  gp[i] = sum_r go[r] (x_ri - x_ri^2),  gb[i] = sum_r go[r] x_ri
// one thread per coordinate i; the sums over r run in order r = 0, 1, ... (FP64 accumulation)
template <typename T>
__global__ void penalized_vjp_kernel(const T* x, const T* g, const T* go, int64_t n, int64_t batch, T* gx, T* gp,
                                     T* gb)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double sp = 0.0, sb = 0.0;
        for (int64_t r = 0; r < batch; ++r) {
            const T w = go[r];
            const T xi = x[r * n + i];
            if (gx) gx[r * n + i] = w * g[r * n + i];
            sp += (double)w * ((double)xi - (double)xi * (double)xi);
            sb += (double)w * (double)xi;
        }
        if (gp) gp[i] = (T)sp;
        if (gb) gb[i] = (T)sb;
    }
}

cudaError_t launch_penalized_vjp(const void* x, const void* g, const void* go, int64_t n, int64_t batch, int dtype,
                                 void* gx, void* gp, void* gb, cudaStream_t s)
{
    const int threads = 256;
    const int64_t want = (n + threads - 1) / threads;
    const int blocks = (int)(want < 4096 ? want : 4096);
    if (dtype == 1)
        penalized_vjp_kernel<double><<<blocks, threads, 0, s>>>((const double*)x, (const double*)g, (const double*)go, n,
                                                                 batch, (double*)gx, (double*)gp, (double*)gb);
    else
        penalized_vjp_kernel<float><<<blocks, threads, 0, s>>>((const float*)x, (const float*)g, (const float*)go, n,
                                                               batch, (float*)gx, (float*)gp, (float*)gb);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t set_smem(size_t smem)
{
    // always opted in: the static shared memory counts against the 48 KB default as well
    return cudaFuncSetAttribute(phase_a_gemv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_phase_a_gemv(int max_ld) { return set_smem<float>((size_t)max_ld * sizeof(float)); }

// persistent grid: every CTA that fits on the GPU at once, never more CTAs than items
template <typename T>
static int grid_for(size_t smem, int nitems)
{
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, phase_a_gemv_kernel<T>, kThreads, smem);
    if (e != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    int g = sms * per;
    return nitems < g ? nitems : g;
}

int gemv_grid(int max_ld, int nitems) { return grid_for<float>((size_t)max_ld * sizeof(float), nitems); }

cudaError_t launch_phase_a_gemv_f32(const TickArgs& a, cudaStream_t s)
{
    // shared: u of the widest lane (ld floats); rows_per_item <= kThreads
    size_t smem = (size_t)a.max_ld * sizeof(float);
    phase_a_gemv_kernel<float><<<a.grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// gradient lanes on the GEMV kernel: shared memory holds one point (n entries of T); the
// queue counters a.work / a.done must be zero (the last CTA leaves them zero again)
cudaError_t launch_phase_a_grad(const TickArgs& a, int dtype, int64_t n, cudaStream_t s)
{
    TickArgs t = a;
    t.fused = 0;
    t.active_count = nullptr;
    if (dtype == 1) {
        const size_t smem = (size_t)n * sizeof(double);
        cudaError_t e = set_smem<double>(smem);
        if (e != cudaSuccess) return e;
        t.grid = grid_for<double>(smem, a.nitems);
        phase_a_gemv_kernel<double><<<t.grid, kThreads, smem, s>>>(t);
    } else {
        const size_t smem = (size_t)n * sizeof(float);
        cudaError_t e = set_smem<float>(smem);
        if (e != cudaSuccess) return e;
        t.grid = grid_for<float>(smem, a.nitems);
        phase_a_gemv_kernel<float><<<t.grid, kThreads, smem, s>>>(t);
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
