// Phase A and the lane update on CUDA cores, persistent lane loop: one launch runs many
// steps of every GEMV lane, and the lanes advance independently of each other.
//
// Work is a global ring of (lane, row block) entries.  A CTA pops the next entry, computes
// that block exactly as the lock-step tick kernel does (same functions, same order of
// operations, so a lane's results do not depend on the scheduler), and counts itself in;
// the CTA that completes a lane's count runs the lane's update and pushes the lane's
// blocks of its next step.  There is no grid-wide barrier between steps: while one lane
// runs its update, the other lanes' blocks keep HBM busy, so the per-step cost of a
// kernel launch, the ramp-up and the update latency of the slowest lane disappears.
//
// A lane stops pushing when it is finished or has used its budget of steps for this
// launch; the last lane to stop pushes one poison entry per CTA and every CTA leaves at
// its poison.  Ring slots carry a sequence number (position / capacity + 1) in their high
// 32 bits, so a consumer that popped position q waits until the slot holds position q's
// entry; every wait gives up after A.wait_ns (5 s unless the caller sets a limit), sets the
// error flag and ends the CTA.  No asynchronous copy is in flight during that wait, so a CTA
// can always leave there; every other CTA then ends at its own next wait.
//
// With symmetric storage (A.sym set) a step that multiplies by Q_off has two stages: one
// entry per kSymGroup stored tiles (entry block < kBlockFlag), whose products go to the lane's partial
// vectors, and then, pushed by the CTA that finished the lane's last tile, one entry per row
// block (kBlockFlag | b) that sums the block's partials and runs the epilogue.  Evaluation
// steps read the dense evaluation matrix and have row-block entries only.
//
// Lanes written by one CTA are read by CTAs on other SMs within the same launch, so this
// file is compiled with plain loads cached in L2 only (-dlcm=cg): no SM may serve a lane
// vector from a stale L1 line.  Q itself never changes and keeps its non-coherent
// streaming loads.
#include "gemv_rows.cuh"

namespace ubqp {

constexpr uint32_t kLaneSkip = 0xFFFEu;            // seeded block of a finished lane
constexpr uint32_t kLanePoison = 0xFFFFu;          // ends the CTA that pops it
constexpr uint32_t kBlockFlag = 0x8000u;           // symmetric storage: a row-block entry

__device__ __forceinline__ unsigned long long ring_seq(unsigned long long pos, unsigned long long cap)
{
    return (pos / cap + 1ull) << 32;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t loop_clock()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Seeds one launch (one CTA): budgets, the count of lanes with work, and the ring entries
// of every lane's current step in the static item order (largest lanes first); finished
// lanes, and slots that a lane's current step does not use, keep their places as skip
// entries.  When no lane has work, one poison entry per CTA follows so that the loop kernel
// ends at once.
__global__ void __launch_bounds__(1024) lane_loop_seed_kernel(LoopArgs A)
{
    __shared__ int s_active;
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) {
        s_active = 0;
        s_base = *A.tail;
        *A.active_after = 0;
    }
    __syncthreads();
    int mine = 0;
    for (int l = threadIdx.x; l < A.nlanes; l += blockDim.x) {
        const bool act = A.lanes[l].st->phase != PH_DONE;
        A.budget_left[l] = act ? A.budget : 0;
        mine += act ? 1 : 0;
    }
    if (mine) atomicAdd(&s_active, mine);
    __syncthreads();
    const unsigned long long base = s_base, cap = A.cap;
    for (int e = threadIdx.x; e < A.nitems; e += blockDim.x) {
        const int2 it = A.items[e];
        const int ph = A.lanes[it.x].st->phase;
        bool act = ph != PH_DONE;
        unsigned blk = (unsigned)it.y;
        if (A.sym && act) {   // a tile step, or an evaluation step (row blocks only)
            const SymLane& S = A.sym[it.x];
            act = it.y < (ph == PH_EVAL ? S.nb : S.ngroups);
            if (ph == PH_EVAL) blk |= kBlockFlag;
        }
        const unsigned long long pos = base + (unsigned long long)e;
        const unsigned long long pay = act ? ((unsigned long long)it.x << 16) | blk
                                           : ((unsigned long long)kLaneSkip << 16);
        A.ring[pos & (cap - 1)] = ring_seq(pos, cap) | pay;
    }
    const int npoison = s_active == 0 ? A.grid : 0;
    for (int e = threadIdx.x; e < npoison; e += blockDim.x) {
        const unsigned long long pos = base + (unsigned long long)A.nitems + e;
        A.ring[pos & (cap - 1)] = ring_seq(pos, cap) | ((unsigned long long)kLanePoison << 16);
    }
    if (threadIdx.x == 0) {
        *A.tail = base + (unsigned long long)A.nitems + (unsigned long long)npoison;
        *A.running = s_active;
    }
}

__global__ void __launch_bounds__(kThreads, 4) lane_loop_kernel(LoopArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* su = reinterpret_cast<float*>(smem_raw);
    __shared__ double sv[kThreads];
    __shared__ unsigned long long s_entry, s_base;
    __shared__ int s_last, s_npush;
    __shared__ unsigned s_pay;
    __shared__ __align__(16) LaneDev sL;   // the popped lane's descriptor
    __shared__ float s_col[kSymGroup][kWarps][kSymT];
    static_assert(sizeof(LaneDev) % 8 == 0, "descriptor copied in 8-byte pieces");
    const unsigned long long cap = A.cap, mask = cap - 1;

    // (Reserving the next position while the current item is processed -- pop-ahead, which the
    // protocol model in tests/test_lane_loop_protocol.py shows deadlock-free -- was measured
    // slower on the 40-lane sweep, 14.9 s against 13.7 s per step: an entry whose position a
    // busy CTA holds waits for that CTA instead of the next idle one.)
    for (;;) {
        // ---- pop the next entry and wait until its slot is written
        if (threadIdx.x == 0) {
            const unsigned long long pos = atomicAdd(A.head, 1ull);
            const unsigned long long want = ring_seq(pos, cap);
            const uint64_t t0 = loop_clock();
            unsigned long long v;
            for (;;) {
                v = ld_acquire(A.ring + (pos & mask));
                if ((v & 0xFFFFFFFF00000000ull) == want) break;
                if (loop_clock() - t0 > A.wait_ns) {
                    atomicExch(A.err, 1);
                    v = (unsigned long long)kLanePoison << 16;
                    break;
                }
                __nanosleep(64);   // idle CTAs poll gently: the ring shares L2 with the rows
            }
            s_entry = v;
        }
        __syncthreads();
        const unsigned pay = (unsigned)(s_entry & 0xFFFFFFFFull);
        const int lane_id = (int)(pay >> 16);
        int blk = (int)(pay & 0xFFFFu);
        if ((unsigned)lane_id == kLanePoison) break;
        if ((unsigned)lane_id == kLaneSkip) {
            __syncthreads();
            continue;
        }

        // ---- one (lane, row block) item, as in the lock-step kernel.  The descriptor never
        // changes, so it comes through the read-only path (cached in L1 across steps).
        if (threadIdx.x < (int)(sizeof(LaneDev) / 8))
            reinterpret_cast<int2*>(&sL)[threadIdx.x] = __ldg(reinterpret_cast<const int2*>(A.lanes + lane_id) + threadIdx.x);
        __syncthreads();
        const LaneDev& L = sL;
        if (A.sym && !(blk & kBlockFlag)) {
            // ---- symmetric storage, stage 1: one tile's row and column products
            const SymLane S = A.sym[lane_id];
            sym_group_item(S, L, blk, s_col, A.P);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                s_npush = 0;
                if (atomicAdd(S.counter, 1u) == (unsigned)(S.ngroups - 1)) {
                    // the lane's last tile: its row blocks come next
                    *S.counter = 0u;
                    s_npush = S.nb;
                    s_pay = ((unsigned)lane_id << 16) | kBlockFlag;
                    s_base = atomicAdd(A.tail, (unsigned long long)S.nb);
                    __threadfence();
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < s_npush; t += kThreads) {
                const unsigned long long pos = s_base + (unsigned long long)t;
                st_release(A.ring + (pos & mask), ring_seq(pos, cap) | s_pay | (unsigned)t);
            }
            __syncthreads();
            continue;
        }
        blk &= ~(int)kBlockFlag;
        const int ph = L.st->phase;
        const int k = L.st->k;
        const int row0 = blk * A.rows_per_item;
        const int rows = min(A.rows_per_item, L.n - row0);
        int sym_parts = 0;
        if (A.sym && ph != PH_EVAL) {
            // ---- symmetric storage, stage 2: the block's products from its partial vectors
            const SymLane S = A.sym[lane_id];
            sym_block_sums(S, L, blk, rows, sv);
            sym_parts = S.nb;
            __syncthreads();
        } else {
            item_load_u(L, su);
            __syncthreads();
            item_rows_solver(L, ph, row0, rows, su, sv, threadIdx.x & 31, threadIdx.x >> 5);
            __syncthreads();
        }
        item_finish(L, ph, k, blk, row0, rows, sv, A.P, sym_parts);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(L.counter, 1u) == (unsigned)(L.nblk - 1));
        __syncthreads();

        // ---- the CTA that completed the step: update, then the lane's next step or its end
        if (s_last) {
            __threadfence();
            lane_update(L, A.P, nullptr);
            __syncthreads();
            if (threadIdx.x == 0) {
                *L.counter = 0u;
                const int left = A.budget_left[lane_id] - 1;
                A.budget_left[lane_id] = left;
                const bool done = L.st->phase == PH_DONE;
                if (!done && left > 0) {
                    // next step: dense row blocks, or with symmetric storage the tiles (the
                    // row blocks alone for an evaluation step)
                    const bool tiles = A.sym && L.st->phase != PH_EVAL;
                    const int cnt = tiles ? A.sym[lane_id].ngroups : L.nblk;
                    s_npush = cnt;
                    s_pay = ((unsigned)lane_id << 16) | (A.sym && !tiles ? kBlockFlag : 0u);
                    s_base = atomicAdd(A.tail, (unsigned long long)cnt);
                } else {
                    if (!done) atomicAdd(A.active_after, 1);
                    const bool last_lane = atomicSub(A.running, 1) == 1;
                    s_npush = last_lane ? (int)gridDim.x : 0;
                    s_pay = kLanePoison << 16;
                    s_base = last_lane ? atomicAdd(A.tail, (unsigned long long)gridDim.x) : 0ull;
                }
                __threadfence();
            }
            __syncthreads();
            const bool poison = s_pay == (kLanePoison << 16);
            for (int t = threadIdx.x; t < s_npush; t += kThreads) {
                const unsigned long long pos = s_base + (unsigned long long)t;
                st_release(A.ring + (pos & mask), ring_seq(pos, cap) | s_pay | (poison ? 0u : (unsigned)t));
            }
        }
        __syncthreads();
    }
}

cudaError_t prepare_lane_loop(int max_ld)
{
    const size_t smem = (size_t)max_ld * sizeof(float);
    // always opted in: the static shared memory counts against the 48 KB default as well
    return cudaFuncSetAttribute(lane_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// CTAs resident at once (the loop's CTAs wait on one another's pushes, so the grid never
// exceeds what the GPU holds)
int lane_loop_grid(int max_ld)
{
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lane_loop_kernel, kThreads,
                                                      (size_t)max_ld * sizeof(float)) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    return sms * per;
}

cudaError_t launch_lane_loop(const LoopArgs& a, cudaStream_t s)
{
    lane_loop_seed_kernel<<<1, 1024, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lane_loop_kernel<<<a.grid, kThreads, (size_t)a.max_ld * sizeof(float), s>>>(a);
    return cudaGetLastError();
}

}  // namespace ubqp
