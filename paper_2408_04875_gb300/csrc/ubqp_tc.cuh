// Tensor-core phase A (tc_gemm.cu): per-instance tile table and launch arguments.
#pragma once

#include <cuda.h>

#include "ubqp_internal.cuh"

namespace ubqp {

constexpr int kTcMaxStages = 4;
constexpr int kTcpMaxStages = 8;   // persistent kernel
constexpr int kTcMaxBn = 128;   // lanes per N tile (UMMA N)
constexpr int kTcMaxCluster = 8;   // CTAs per split-K cluster

// One instance of the batched path: BF16 Q_off (ld x ld) and its lanes' packed inputs
// (hi and lo terms, R rows of ld), with the TMA descriptors of all three.
struct alignas(128) TcInst {
    CUtensorMap tmA;     // Q_off in the tiled layout (qbf_index): a (ld*ld/64) x 64 view,
                         // box 64 x 128 = one contiguous 16 KB tile
    CUtensorMap tmBhi;   // lane inputs (hi term), box 64 x bn
    CUtensorMap tmBlo;   // lane inputs (lo term), box 64 x bn
    int32_t n, ld, R, lane0;
    int32_t m_tiles, n_tiles, bn, two_terms;
    int32_t cluster0;    // first cluster of this instance in the launch
    int32_t pad_;
    const int32_t* nt_active;   // per N tile: unfinished lanes (null: scan the lane states)
};

struct TcArgs {
    const TcInst* inst;
    int32_t ninst;
    int32_t stages;
    int32_t tmem_cols;
    int32_t max_bn;
    int32_t two_any;     // some instance carries the lo term (shared-memory sizing)
    const LaneDev* lanes;
    float* raw;          // probe mode: D written as [lane][row] (ld stride) instead of the epilogue
    int32_t* err;        // set when a bounded wait ran out
    unsigned long long* flops;  // algorithmic flops of the tiles computed (may be null)
    int32_t fuse;        // 1: the warp that finishes a lane's last M tile runs its update
                         // (every lane has at most 32 M tiles); 0: a separate update launch
    int32_t* active_count;  // fused: incremented by every lane still active after its update
    Params P;
};

size_t tc_smem_bytes(int bn, bool two, int stages);
int tc_pick_stages(int bn, bool two);
cudaError_t tc_launch(const TcArgs& a, int total_clusters, int S, cudaStream_t st);
int tc_max_active_clusters(int bn, bool two, int stages, int S);
int tc_tmem_cols(int bn, bool two);
CUresult tc_encode_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows);

// persistent kernel (many tiles, no split-K)
size_t tcp_smem_bytes(int bn, bool two, int stages);
int tcp_pick_stages(int bn, bool two);
int tcp_tmem_cols(bool two);
int tcp_grid(const TcArgs& a, int ntiles);
cudaError_t tcp_launch(const TcArgs& a, int ntiles, int grid, cudaStream_t st);

// cluster size for a launch of `tiles` output tiles: the largest S <= 8 such that every
// cluster is resident at once, one CTA per SM, and each CTA keeps >= 2 k-blocks
int tc_pick_cluster(int tiles, int kb_min, int bn, bool two, int stages, int num_sms);

}  // namespace ubqp
