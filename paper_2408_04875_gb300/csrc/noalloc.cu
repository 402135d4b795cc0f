// ubqp_penalized_eval_noalloc: the penalized objective and its gradient for callers that
// must not allocate device memory.  Some callers manage every byte of device memory
// through their own pool or a fixed budget and may not call cudaMalloc/cudaFree (which
// can also synchronize the whole device); this entry point gives them the same
// computation as ubqp_penalized_eval, with the same kernel and the same work partition,
// with its scratch in a fixed static device array.
//
// The scratch (per-point descriptors, work items, the work-queue counters, per-block
// partial sums) lives in g_noalloc_scratch below.  Every GPU that loads the library holds
// it until the process exits.  All calls share it and it keeps the last call's contents;
// each call rewrites every byte it later reads (the queue counters are cleared by the
// call's set-up kernel), so nothing has to start at zero.  Calls that overlap on the GPU
// (other streams, other host threads) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/ubqp.h"
#include "ubqp_internal.cuh"

namespace ubqp {

constexpr int kNoallocMaxLanes = 256;
constexpr int kNoallocMaxItems = 16384;
constexpr size_t kLanesBytes = (size_t)kNoallocMaxLanes * 320;   // room for one descriptor per point
static_assert(sizeof(LaneDev) <= 320, "descriptor outgrew its scratch slot");
constexpr size_t kItemsBytes = (size_t)kNoallocMaxItems * sizeof(int2);
constexpr size_t kQueueBytes = 256;
constexpr size_t kPartBytes = (size_t)kNoallocMaxItems * sizeof(Partial);
constexpr size_t kLanesOff = 0;
constexpr size_t kItemsOff = (kLanesBytes + 255) / 256 * 256;
constexpr size_t kQueueOff = kItemsOff + (kItemsBytes + 255) / 256 * 256;
constexpr size_t kPartOff = kQueueOff + kQueueBytes;
constexpr size_t kScratchBytes = kPartOff + kPartBytes;
static_assert(kScratchBytes == UBQP_NOALLOC_SCRATCH_BYTES, "header and scratch layout disagree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch in each CUDA context that has used this entry point.
// The key is the context's unique ID (cuCtxGetId), not the device index: after a device
// reset the runtime creates a new primary context, reloads the module, and the array may
// live at another address; the new context has a new ID, so its address is resolved again.
typedef CUresult (*PFN_ctx_current)(CUcontext*);
typedef CUresult (*PFN_ctx_id)(CUcontext, unsigned long long*);

static std::mutex g_noalloc_mu;
struct ScratchAddr {
    unsigned long long ctx_id;
    void* addr;
};
static ScratchAddr g_noalloc_addr[64];
static int g_noalloc_next = 0;

template <class F>
static F driver_fn(const char* name)
{
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return reinterpret_cast<F>(p);
}

static cudaError_t noalloc_scratch(void** out)
{
    static PFN_ctx_current ctx_current = driver_fn<PFN_ctx_current>("cuCtxGetCurrent");
    static PFN_ctx_id ctx_id = driver_fn<PFN_ctx_id>("cuCtxGetId");
    if (!ctx_current || !ctx_id) return cudaErrorNotSupported;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (ctx_current(&ctx) == CUDA_SUCCESS && !ctx) {
        // no context current on this thread yet: make the device's primary context current
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (ctx_current(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    }
    if (!ctx || ctx_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    cudaError_t e;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (const ScratchAddr& a : g_noalloc_addr)
        if (a.addr && a.ctx_id == id) {
            *out = a.addr;
            return cudaSuccess;
        }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[g_noalloc_next] = ScratchAddr{id, p};
    g_noalloc_next = (g_noalloc_next + 1) % 64;
    *out = p;
    return cudaSuccess;
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
    clear_error();
    if (!Q || !x || n < 1 || batch < 1 || (dtype != UBQP_DTYPE_F32 && dtype != UBQP_DTYPE_F64)) {
        set_error("ubqp_penalized_eval_noalloc: need Q, x, n >= 1, batch >= 1 and dtype UBQP_DTYPE_F32 or _F64");
        return UBQP_EINVAL;
    }
    const int64_t es = dtype == UBQP_DTYPE_F64 ? 8 : 4;
    // limits of the static scratch and of shared memory
    if (batch > kNoallocMaxLanes) {
        set_error("ubqp_penalized_eval_noalloc: batch = %lld exceeds the scratch limit of %d points", (long long)batch,
                  kNoallocMaxLanes);
        return UBQP_EINVAL;
    }
    if (n * es > 200 * 1024) {
        set_error("ubqp_penalized_eval_noalloc: n * element size = %lld bytes exceeds the limit of 200 KiB",
                  (long long)(n * es));
        return UBQP_EINVAL;
    }
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("ubqp_penalized_eval_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
        return UBQP_ECUDA;
    }
    // the work partition of ubqp_penalized_eval (same rows per item), so both return the same values
    int rb = 8;
    while (rb < 256 && batch * n / rb > 8 * (int64_t)sms) rb *= 2;
    const int64_t nblk = (n + rb - 1) / rb;
    if (batch * nblk > kNoallocMaxItems) {
        set_error("ubqp_penalized_eval_noalloc: batch * ceil(n / %d) = %lld work items exceeds the limit of %d", rb,
                  (long long)(batch * nblk), kNoallocMaxItems);
        return UBQP_EINVAL;
    }
    const void* ptrs[6] = {Q, b, p, x, h_out, g_out};
    for (const void* q : ptrs) {
        if (q && (reinterpret_cast<uintptr_t>(q) % (uintptr_t)es) != 0) {
            set_error("ubqp_penalized_eval_noalloc: every pointer must be aligned to its element size");
            return UBQP_EINVAL;
        }
        if (q && !on_device(q)) {
            set_error("ubqp_penalized_eval_noalloc: all pointers must be device memory");
            return UBQP_EINVAL;
        }
    }
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) {
        set_error("ubqp_penalized_eval_noalloc: resolving the scratch array failed: %s", cudaGetErrorString(e));
        return UBQP_ECUDA;
    }
    unsigned char* base = static_cast<unsigned char*>(scratch);
    cudaStream_t s = (cudaStream_t)stream;
    const int nitems = (int)(batch * nblk);
    e = launch_grad_setup(reinterpret_cast<LaneDev*>(base + kLanesOff), reinterpret_cast<int2*>(base + kItemsOff),
                          reinterpret_cast<int32_t*>(base + kQueueOff), reinterpret_cast<Partial*>(base + kPartOff), Q, b,
                          p, x, g_out, (int)n, (int)batch, (int)nblk, (int)es, s);
    TickArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.lanes = reinterpret_cast<const LaneDev*>(base + kLanesOff);
    ta.items = reinterpret_cast<const int2*>(base + kItemsOff);
    ta.nitems = nitems;
    ta.rows_per_item = rb;
    ta.nlanes = (int)batch;
    ta.max_ld = (int)n;
    ta.work = reinterpret_cast<int32_t*>(base + kQueueOff);
    ta.done = ta.work + 1;
    if (e == cudaSuccess) e = launch_phase_a_grad(ta, dtype, n, s);
    if (e == cudaSuccess && h_out) e = launch_grad_reduce(ta.lanes, (int)batch, h_out, dtype, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("ubqp_penalized_eval_noalloc: %s", cudaGetErrorString(e));
        return UBQP_ECUDA;
    }
    return UBQP_OK;
}
