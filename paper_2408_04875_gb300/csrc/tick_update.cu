// Phase B as a stand-alone kernel: one CTA per lane runs lane_update (lane_update.cuh).
// Used for tensor-core lanes; GEMV lanes run the same update inside the fused tick.
#include "lane_update.cuh"

namespace ubqp {

__global__ void __launch_bounds__(kBThreads) phase_b_kernel(TickArgs A, int32_t* active_count)
{
    lane_update<true>(A.lanes[blockIdx.x], A.P, active_count);
}

// CTA size: each update is a chain of dependent steps (partials, decision, element-wise
// pass), so throughput comes from many updates in flight.  About three 256-thread CTAs fit
// on an SM; beyond one such wave of lanes, smaller CTAs let more updates overlap.
static int phase_b_threads(int nlanes)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
    }
    if (nlanes <= 3 * sms) return kBThreads;
    if (nlanes <= 6 * sms) return kBThreads / 2;
    return kBThreads / 4;
}

cudaError_t launch_phase_b(const TickArgs& a, int32_t* active_count, cudaStream_t s)
{
    phase_b_kernel<<<a.nlanes, phase_b_threads(a.nlanes), 0, s>>>(a, active_count);
    return cudaGetLastError();
}

}  // namespace ubqp
