// ubqp_penalized_eval_noalloc: the penalized objective and its gradient for callers that
// must not allocate device memory.  Some callers manage every byte of device memory
// through their own pool or a fixed budget and may not call cudaMalloc/cudaFree (which
// can also synchronize the whole device); this entry point gives them the same
// computation as ubqp_penalized_eval with its scratch in a fixed static device array.
//
// The scratch (per-point descriptors, work items, per-block partial sums) lives in
// g_noalloc_scratch below.  Every GPU that loads the library holds it until the process
// exits.  All calls share it and it keeps the last call's contents; each call rewrites
// every byte it later reads, so nothing has to start at zero.  Calls that overlap on
// the GPU (other streams, other host threads) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/ubqp.h"
#include "ubqp_internal.cuh"

namespace ubqp {

constexpr int kNoallocMaxLanes = 256;
constexpr int kNoallocMaxItems = 16384;
constexpr size_t kLanesBytes = (size_t)kNoallocMaxLanes * 256;   // room for one descriptor per point
static_assert(sizeof(LaneDev) <= 256, "descriptor outgrew its scratch slot");
constexpr size_t kItemsBytes = (size_t)kNoallocMaxItems * sizeof(int2);
constexpr size_t kPartBytes = (size_t)kNoallocMaxItems * sizeof(Partial);
constexpr size_t kLanesOff = 0;
constexpr size_t kItemsOff = (kLanesBytes + 255) / 256 * 256;
constexpr size_t kPartOff = kItemsOff + (kItemsBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kPartOff + kPartBytes;
static_assert(kScratchBytes == UBQP_NOALLOC_SCRATCH_BYTES, "header and scratch layout disagree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of g_noalloc_scratch, resolved once per device with that device current
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[128];

static cudaError_t noalloc_scratch(int dev, void** out)
{
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

// descriptors and work items of `batch` gradient lanes, written on the device
__global__ void noalloc_setup_kernel(unsigned char* scratch, const void* Q, const void* b, const void* p,
                                     const void* x, void* g, int n, int batch, int nblk, int es)
{
    LaneDev* lanes = reinterpret_cast<LaneDev*>(scratch + kLanesOff);
    int2* items = reinterpret_cast<int2*>(scratch + kItemsOff);
    Partial* part = reinterpret_cast<Partial*>(scratch + kPartOff);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
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

static bool on_device(const void* ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace ubqp

using namespace ubqp;

extern "C" int ubqp_penalized_eval_noalloc(const void* Q, const void* b, const void* p, const void* x, int64_t n,
                                           int64_t batch, int dtype, void* h_out, void* g_out, void* stream)
{
    if (!Q || !x || n < 1 || batch < 1 || (dtype != UBQP_DTYPE_F32 && dtype != UBQP_DTYPE_F64)) return UBQP_EINVAL;
    const size_t es = dtype == UBQP_DTYPE_F64 ? 8 : 4;
    // limits of the static scratch: batch <= 256 points and batch * ceil(n / rows) <= 16384
    // blocks with at most 256 rows per block; u of one point must fit in shared memory
    if (batch > kNoallocMaxLanes || n * (int64_t)es > 200 * 1024) return UBQP_EINVAL;
    int rb = 16;
    while (rb < 256 && batch * ((n + rb - 1) / rb) > kNoallocMaxItems) rb *= 2;
    const int64_t nblk = (n + rb - 1) / rb;
    if (batch * nblk > kNoallocMaxItems) return UBQP_EINVAL;
    if (!on_device(Q) || !on_device(x) || (b && !on_device(b)) || (p && !on_device(p)) ||
        (h_out && !on_device(h_out)) || (g_out && !on_device(g_out)))
        return UBQP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return UBQP_ECUDA;
    void* scratch = nullptr;
    if (noalloc_scratch(dev, &scratch) != cudaSuccess) return UBQP_ECUDA;
    unsigned char* base = static_cast<unsigned char*>(scratch);
    cudaStream_t s = (cudaStream_t)stream;
    const int nitems = (int)(batch * nblk);
    noalloc_setup_kernel<<<(nitems + 255) / 256, 256, 0, s>>>(base, Q, b, p, x, g_out, (int)n, (int)batch,
                                                               (int)nblk, (int)es);
    cudaError_t e = cudaGetLastError();
    TickArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.lanes = reinterpret_cast<const LaneDev*>(base + kLanesOff);
    ta.items = reinterpret_cast<const int2*>(base + kItemsOff);
    ta.nitems = nitems;
    ta.rows_per_item = rb;
    ta.nlanes = (int)batch;
    ta.max_ld = (int)n;
    if (e == cudaSuccess) e = launch_phase_a_grad(ta, dtype, n, s);
    if (e == cudaSuccess && h_out) e = launch_grad_reduce(ta.lanes, (int)batch, h_out, dtype, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? UBQP_OK : UBQP_ECUDA;
}
