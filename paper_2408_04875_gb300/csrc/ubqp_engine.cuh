// Host-side engine structures shared by the set-up kernels and the driver.
#pragma once

#include "ubqp_internal.cuh"

namespace ubqp {

// Layout of the BF16 matrix of the tensor-core path: tiles of 128 rows x 64 columns (one
// k-block of one M tile), stored contiguously in the order [M tile][k-block], rows of 64
// entries inside a tile.  One TMA box is then one contiguous 16 KB run of memory.
__host__ __device__ __forceinline__ size_t qbf_index(size_t i, size_t j, size_t ld)
{
    return (((i >> 7) * (ld >> 6) + (j >> 6)) * 128 + (i & 127)) * 64 + (j & 63);
}

struct RefArgs {
    int32_t n, ld, inst, diag_only_mu;
    int32_t no_gamma;       // Q, b are already Q', b' (test entries): gamma = 0
    int32_t pad_;
    const double* Q;        // n x n original (device)
    const double* b;        // n or null
    const double* mu;       // n x n or null
    double sigma;           // std-dev of drawn perturbation (0 = none)
    double margin;
    uint64_t seed;
    float* Qoff;            // GEMV: n x ld FP32 (or null)
    __nv_bfloat16* Qbf;     // TC: ld x ld BF16 in the tiled layout of qbf_index (or null)
    float2* Qeval;          // GEMV: n x ld original as (hi, lo) FP32 pairs (or null)
    float *d, *bprime, *oabs, *rabs, *tsum;   // tsum = d + b' formed in FP64
    double *borig, *qdb, *gamma;
    float* scal;            // [0] max_{i!=j} |Q'_ij| stored, [1] max rabs
    int* inexact;           // TC: set when BF16 changed an off-diagonal entry
};

// validation of one instance: out[0] = max |Q_ij - Q_ji|, out[1] = max off-diagonal |Q_ij|,
// out[2] = non-finite flag, out[3] = max |Q_ij|
struct ValArgs {
    const double* Q;
    const double* b;
    float* out;
    unsigned long long* nnz;   // stored off-diagonal entries (nonzero Q_ij, i != j)
    int32_t n, pad_;
};

struct LaneInit {
    int32_t phase;          // first phase (JACOBI, EVAL or INNER)
    int32_t start_kind;     // 0 = 0.5 (Jacobi guess), 1 = drawn uniform start
    int32_t inst, restart;
    const double* x0;       // explicit start (device) or null
    const double* p0;       // explicit penalty (device) or null
};

struct LaneInitArgs {
    const LaneDev* lanes;
    const LaneInit* init;
    uint64_t seed;
};

struct FinalArgs {
    const LaneDev* lanes;
    const int32_t* lane0;
    const int32_t* nlanes;
    double* obj;
    int32_t* best_lane;
    uint8_t* const* x_out;  // device pointers, one per instance
};

// Q'_off rows -> symmetric storage tiles (ld a multiple of 128)
cudaError_t launch_pack_sym(const float* Qoff, int n, int ld, float* Qsym, cudaStream_t s);

// one launch for every instance of a batch; row0[t] = first global row of instance t
cudaError_t launch_validate(const ValArgs* v, const int64_t* row0, int ninst, int64_t rows, cudaStream_t s);
cudaError_t launch_reformulate(const RefArgs* args, const int64_t* row0, int ninst, int64_t rows, cudaStream_t s);
cudaError_t launch_sell_width(const float* Qoff, int n, int ld, int32_t* width, cudaStream_t s);
cudaError_t launch_sell_pack(const float* Qoff, int n, int ld, const int64_t* spo, float* vals, uint16_t* cols,
                             cudaStream_t s);
cudaError_t launch_count_offdiag(const double* Q, int n, unsigned long long* out, cudaStream_t s);
cudaError_t launch_lane_init(const LaneInitArgs& a, int nlanes, cudaStream_t s);
cudaError_t launch_finalize(const FinalArgs& a, int ninst, cudaStream_t s);
cudaError_t launch_lane_vec_to_f64(const LaneDev* lanes, int lane, int v, int n, double* out, cudaStream_t s);
cudaError_t launch_trace_to_f64(const float* in, double* out, int64_t count, cudaStream_t s);

// tensor-core phase A (tc_gemm.cu)
struct TcInst;
cudaError_t launch_phase_a_tc(const TcInst* insts_dev, int ninst_tc, int total_ctas, const LaneDev* lanes,
                              Params P, int cluster_k, cudaStream_t s);

}  // namespace ubqp
