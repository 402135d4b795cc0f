// Phase B as a stand-alone kernel: one CTA per lane runs lane_update (lane_update.cuh).
// Used for tensor-core lanes; GEMV lanes run the same update inside the fused tick.
#include "lane_update.cuh"

namespace ubqp {

__global__ void __launch_bounds__(kBThreads) phase_b_kernel(TickArgs A, int32_t* active_count)
{
    lane_update(A.lanes[blockIdx.x], A.P, active_count);
}

cudaError_t launch_phase_b(const TickArgs& a, int32_t* active_count, cudaStream_t s)
{
    phase_b_kernel<<<a.nlanes, kBThreads, 0, s>>>(a, active_count);
    return cudaGetLastError();
}

}  // namespace ubqp
