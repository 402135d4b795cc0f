// Host driver and C ABI of the vectorized PSDP solver (see include/ubqp.h).
//
// One call = one Solver: stage the inputs on the device, validate them, reformulate
// every instance (Sec. 3.5), lay out one lane per (instance, start), then advance all
// lanes in ticks (phase A matvec + phase B update) until every lane is done.  Ticks are
// enqueued in batches captured once into a CUDA graph; the host only reads one counter
// per batch.  Finally the best lane of every instance is selected on the device and its
// rounded point and exact objective are returned.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ubqp.h"
#include "ubqp_engine.cuh"
#include "ubqp_tc.cuh"

namespace ubqp {

static thread_local char g_last_error[512] = "";
static thread_local std::vector<float> g_tl_ms;
static thread_local std::vector<int64_t> g_tl_work;

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

void clear_error() { g_last_error[0] = 0; }

#define UBQP_CK(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? UBQP_ENOMEM : UBQP_ECUDA;               \
        }                                                                                    \
    } while (0)

static bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// a stream-ordered temporary that is freed on every early return; the success path frees
// it itself and then calls release()
struct AsyncTemp {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    AsyncTemp() = default;
    AsyncTemp(const AsyncTemp&) = delete;
    AsyncTemp& operator=(const AsyncTemp&) = delete;
    ~AsyncTemp()
    {
        if (p) cudaFreeAsync(p, s);
    }
    void hold(void* ptr, cudaStream_t stream)
    {
        p = ptr;
        s = stream;
    }
    void release() { p = nullptr; }
};

// one device allocation carved into 256-byte aligned pieces
class Arena {
  public:
    size_t reserve(size_t bytes)
    {
        size_t off = size_;
        size_ += round_up(bytes ? bytes : 1, 256);
        return off;
    }
    int commit()
    {
        if (size_ == 0) return UBQP_OK;
        cudaError_t e = cudaMalloc(&base_, size_);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of %zu bytes failed: %s", size_, cudaGetErrorString(e));
            base_ = nullptr;
            return e == cudaErrorMemoryAllocation ? UBQP_ENOMEM : UBQP_ECUDA;
        }
        return UBQP_OK;
    }
    template <class T>
    T* at(size_t off) const
    {
        return reinterpret_cast<T*>(static_cast<char*>(base_) + off);
    }
    size_t size() const { return size_; }
    ~Arena()
    {
        if (base_) cudaFree(base_);
    }

  private:
    void* base_ = nullptr;
    size_t size_ = 0;
};

static Params make_params(const ubqp_opts& o, int64_t* hist)
{
    Params P;
    P.max_outer = o.max_outer;
    P.max_inner = o.max_inner;
    P.lob_max = o.lobpcg_max_iter;
    P.jac_max = o.jacobi_max_iter;
    P.tol_inner = (float)o.tol_inner;
    P.tol_outer = (float)o.tol_outer;
    P.eta = (float)o.eta;
    P.alpha_min = (float)o.alpha_min;
    P.alpha_max = (float)o.alpha_max;
    P.tau_z = (float)o.tau_z;
    P.eps_hp_rel = (float)o.eps_hp_rel;
    P.lambda_floor_rel = (float)o.lambda_floor_rel;
    // the Ritz value approaches lambda_min from above, so a loose stop overstates alpha of
    // Eq. (eq:alpha1); tensor-core lanes stop at their BF16 x2 products' resolution at most
    P.lob_tol = (float)(o.precision == UBQP_FP32 ? o.lobpcg_tol : std::max(o.lobpcg_tol, 1e-5));
    P.jac_tol = 2e-7f;
    P.hist = hist;
    P.bytes = nullptr;
    return P;
}

static int check_opts(const ubqp_opts& o)
{
    if (o.method != UBQP_PABB && o.method != UBQP_PPA) { set_error("method must be UBQP_PABB or UBQP_PPA"); return UBQP_EINVAL; }
    if (o.max_outer < 0 || o.max_inner < 0) { set_error("max_outer/max_inner must be >= 0"); return UBQP_EINVAL; }
    if (!(o.eta > 0.0 && o.eta < 1.0)) { set_error("eta must lie in (0, 1) (Eq. (eq:alpha1))"); return UBQP_EINVAL; }
    if (!(o.tol_inner > 0.0) || !(o.tol_outer >= 0.0)) { set_error("tolerances must be positive"); return UBQP_EINVAL; }
    if (!(o.alpha_min > 0.0) || !(o.alpha_max >= o.alpha_min)) { set_error("bad BB step clamp"); return UBQP_EINVAL; }
    if (o.restarts < 0 || o.restarts > 4096) { set_error("restarts must be in [0, 4096]"); return UBQP_EINVAL; }
    if (o.restarts == 0 && o.x_starts) { set_error("the restart tuner (restarts = 0) draws its own starts"); return UBQP_EINVAL; }
    if (o.precision != UBQP_FP32 && o.precision != UBQP_BF16X2_TC && o.precision != UBQP_BF16_TC) {
        set_error("unknown precision");
        return UBQP_EINVAL;
    }
    if (o.lobpcg_max_iter < 1 || o.jacobi_max_iter < 1) { set_error("iteration caps must be >= 1"); return UBQP_EINVAL; }
    if (o.max_ticks_per_sync < 1 || o.max_ticks_per_sync > 4096) { set_error("max_ticks_per_sync out of range"); return UBQP_EINVAL; }
    if (!(o.sigma_rel >= 0.0) || !(o.gamma_margin > 0.0)) { set_error("sigma_rel >= 0 and gamma_margin > 0 required"); return UBQP_EINVAL; }
    if (o.tc_cluster < 0 || o.tc_cluster > 8) { set_error("tc_cluster must be in [0, 8]"); return UBQP_EINVAL; }
    if (o.gemv_kernel < 0 || o.gemv_kernel > 3) { set_error("gemv_kernel must be 0, 1, 2 or 3"); return UBQP_EINVAL; }
    if (o.lane_budget < 0) { set_error("lane_budget must be >= 0"); return UBQP_EINVAL; }
    if (o.wait_limit_us < 0) { set_error("wait_limit_us must be >= 0"); return UBQP_EINVAL; }
    if (o.tc_fuse != 0 && o.tc_fuse != 1) { set_error("tc_fuse must be 0 or 1"); return UBQP_EINVAL; }
    if (o.sparse_storage < 0 || o.sparse_storage > 2) { set_error("sparse_storage must be 0, 1 or 2"); return UBQP_EINVAL; }
    if (o.rows_per_item != 0 && (o.rows_per_item < 8 || o.rows_per_item > 256 || o.rows_per_item % 8 != 0)) {
        set_error("rows_per_item must be 0 or a multiple of 8 in [8, 256]");
        return UBQP_EINVAL;
    }
    return UBQP_OK;
}

// ---------------------------------------------------------------------------------
struct InstIn {
    int64_t n;
    const double* Q;
    const double* b;
    const double* mu;
    const double* starts;   // (R-1) x n extra starts or null
    bool reformulated;      // Q, b are already Q', b' (test entries): no gamma, no mu
};

struct LaneIn {
    int inst, restart, phase, start_kind;
    const double* x0;       // host or device, n doubles, or null
    const double* p0;
    int stop_after, trace_len;
};

struct InstDev {
    int64_t n;
    int ld;
    const double *Q, *b, *mu, *starts;
    size_t o_Q, o_b, o_mu, o_starts;  // staging offsets (when host data)
    bool Q_host, b_host, mu_host, starts_host;
    size_t o_Qoff, o_Qbf, o_Qeval, o_d, o_bp, o_oabs, o_rabs, o_tsum, o_borig, o_qdb, o_gamma;
    size_t ntact = 0;     // TC: index of this instance's first N tile in the active-lane counters
    int nb = 0;           // row blocks of kSymT rows (symmetric storage)
    size_t o_Qsym = 0;    // symmetric storage tiles
    size_t o_Uhi, o_Ulo;
    size_t o_spv = 0, o_spc = 0, o_spo = 0;   // sliced storage (in the second allocation)
    int bn, n_tiles, rows_b;   // tensor-core tiling of this instance's lanes
    int lane0, nl;
};

// ---------------------------------------------------------------------------------
// Measured choice of the tensor-core launch form, cached per shape.  Key: compute capability,
// SM count, output tiles, smallest k-block count, widest N tile, terms, instances and widest
// ld.  Value: the split-K cluster size S (1..8) or 0 for the persistent many-tile kernel.  The
// cache lives in this process; when the environment variable UBQP_TUNE_CACHE names a file, it
// is also read from and written back to that file (one JSON object of "key": value pairs).
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;
static std::string g_tune_file_loaded;

static void tune_load_file_locked(const char* path)
{
    if (!path || g_tune_file_loaded == path) return;
    g_tune_file_loaded = path;
    FILE* f = fopen(path, "r");
    if (!f) return;
    std::string txt;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, k);
    fclose(f);
    // "key": value pairs; keys hold no quotes
    size_t pos = 0;
    for (;;) {
        const size_t a = txt.find('"', pos);
        if (a == std::string::npos) break;
        const size_t b = txt.find('"', a + 1);
        if (b == std::string::npos) break;
        const size_t c = txt.find(':', b + 1);
        if (c == std::string::npos) break;
        char* end = nullptr;
        const long v = strtol(txt.c_str() + c + 1, &end, 10);
        if (end && end != txt.c_str() + c + 1) g_tune[txt.substr(a + 1, b - a - 1)] = (int)v;
        pos = end ? (size_t)(end - txt.c_str()) : b + 1;
    }
}

static void tune_save_file_locked(const char* path)
{
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto& kv : g_tune) fprintf(f, " \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < g_tune.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

class Solver {
  public:
    Solver(const ubqp_opts& o) : o_(o) {}
    ~Solver()
    {
        if (gexec_) cudaGraphExecDestroy(gexec_);
        if (graph_) cudaGraphDestroy(graph_);
        if (h_active_) cudaFreeHost(h_active_);
        if (ev0_) cudaEventDestroy(ev0_);
        if (ev1_) cudaEventDestroy(ev1_);
        for (auto e : evA_) cudaEventDestroy(e);
        if (stream_) {
            cudaStreamSynchronize(stream_);
            cudaStreamDestroy(stream_);
        }
    }

    int setup(const std::vector<InstIn>& insts, const std::vector<LaneIn>& lanes, bool tc)
    {
        tc_ = tc;
        int rc = check_opts(o_);
        if (rc) return rc;
        UBQP_CK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
        cudaStream_t user = (cudaStream_t)o_.stream;
        {
            cudaEvent_t e;
            UBQP_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            cudaEventRecord(e, user);
            cudaStreamWaitEvent(stream_, e, 0);
            cudaEventDestroy(e);
        }
        UBQP_CK(cudaEventCreate(&ev0_));
        UBQP_CK(cudaEventCreate(&ev1_));
        int dev = 0;
        UBQP_CK(cudaGetDevice(&dev));
        UBQP_CK(cudaDeviceGetAttribute(&num_sms_, cudaDevAttrMultiProcessorCount, dev));

        // ---- sliced row storage of Q'_off (sparse data): the stored off-diagonal entries of
        // every instance are counted here, before the layout; the storage is used when they take
        // fewer bytes (4-byte value + 2-byte column) than the symmetric tiles would (2 bytes per
        // matrix entry), or when asked for
        sparse_ = false;
        if (!tc && o_.sparse_storage != 2) {
            std::vector<unsigned long long> cnt(insts.size(), 0);
            unsigned long long* dcnt = nullptr;
            AsyncTemp guard;
            bool any_dev = false;
            for (size_t t = 0; t < insts.size(); ++t) {
                const InstIn& in = insts[t];
                if (is_device_ptr(in.Q)) {
                    any_dev = true;
                    continue;
                }
                unsigned long long c = 0;
                for (int64_t i = 0; i < in.n; ++i)
                    for (int64_t j = 0; j < in.n; ++j) c += (i != j && in.Q[i * in.n + j] != 0.0) ? 1ull : 0ull;
                cnt[t] = c;
            }
            if (any_dev) {
                UBQP_CK(cudaMallocAsync((void**)&dcnt, insts.size() * sizeof(unsigned long long), stream_));
                guard.hold(dcnt, stream_);
                UBQP_CK(cudaMemsetAsync(dcnt, 0, insts.size() * sizeof(unsigned long long), stream_));
                for (size_t t = 0; t < insts.size(); ++t)
                    if (is_device_ptr(insts[t].Q)) UBQP_CK(launch_count_offdiag(insts[t].Q, (int)insts[t].n, dcnt + t, stream_));
                std::vector<unsigned long long> dv(insts.size(), 0);
                UBQP_CK(cudaMemcpyAsync(dv.data(), dcnt, insts.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                        stream_));
                UBQP_CK(cudaStreamSynchronize(stream_));
                for (size_t t = 0; t < insts.size(); ++t)
                    if (is_device_ptr(insts[t].Q)) cnt[t] = dv[t];
                guard.release();
                UBQP_CK(cudaFreeAsync(dcnt, stream_));
            }
            double by_sparse = 0.0, by_sym = 0.0;
            for (size_t t = 0; t < insts.size(); ++t) {
                by_sparse += 6.0 * (double)cnt[t];
                by_sym += 2.0 * (double)insts[t].n * (double)insts[t].n;
            }
            sparse_ = o_.sparse_storage == 1 || by_sparse < by_sym;
        }
        // ---- symmetric storage: only with the lane loop (decided here because it fixes the
        // row padding and the row blocks); tiles are indexed in 15 bits per lane
        if (!sparse_) {
            const bool loop_likely =
                !tc && lanes.size() < 0xFFFEu &&
                (o_.gemv_kernel == 2 || (o_.gemv_kernel == 0 && o_.profile_kernels < 2 && lanes.size() >= 4));
            sym_ = loop_likely && o_.sym_storage != 0;
            for (const InstIn& in : insts) {
                const int64_t nb = (in.n + kSymT - 1) / kSymT;
                if (nb * (nb + 1) / 2 >= 0x8000) sym_ = false;
            }
        }
        // ---- layout
        inst_.resize(insts.size());
        int max_ld = 32;
        for (size_t t = 0; t < insts.size(); ++t) {
            const InstIn& in = insts[t];
            InstDev& I = inst_[t];
            I.n = in.n;
            I.ld = (int)round_up((size_t)in.n, sym_ ? kSymT : (tc ? 128 : 32));
            max_ld = std::max(max_ld, I.ld);
            const size_t n = (size_t)in.n, ld = (size_t)I.ld;
            I.Q_host = !is_device_ptr(in.Q);
            I.b_host = in.b && !is_device_ptr(in.b);
            I.mu_host = in.mu && !is_device_ptr(in.mu);
            I.starts_host = in.starts && !is_device_ptr(in.starts);
            I.o_Q = I.Q_host ? ar_.reserve(n * n * 8) : 0;
            I.o_b = I.b_host ? ar_.reserve(n * 8) : 0;
            I.o_mu = I.mu_host ? ar_.reserve(n * n * 8) : 0;
            I.o_starts = 0;
            I.o_Qoff = tc ? 0 : ar_.reserve(n * ld * 4);
            I.o_Qbf = tc ? ar_.reserve(ld * ld * 2) : 0;
            I.o_Qeval = tc ? 0 : ar_.reserve(n * ld * 8);
            I.nb = (int)(ld / kSymT);
            I.o_Qsym = sym_ ? ar_.reserve((size_t)I.nb * (I.nb + 1) / 2 * kSymT * kSymT * 4) : 0;
            I.o_d = ar_.reserve(ld * 4);
            I.o_bp = ar_.reserve(ld * 4);
            I.o_oabs = ar_.reserve(ld * 4);
            I.o_rabs = ar_.reserve(ld * 4);
            I.o_tsum = ar_.reserve(ld * 4);
            I.o_borig = ar_.reserve(ld * 8);
            I.o_qdb = ar_.reserve(ld * 8);
            I.o_gamma = ar_.reserve(ld * 8);
            I.lane0 = -1;
            I.nl = 0;
        }
        max_ld_ = max_ld;
        o_scal_ = ar_.reserve(insts.size() * 4 * sizeof(float));
        o_row0_ = ar_.reserve((insts.size() + 1) * sizeof(int64_t));
        o_valargs_ = ar_.reserve(insts.size() * sizeof(ValArgs));
        o_refargs_ = ar_.reserve(insts.size() * sizeof(RefArgs));
        o_valid_ = ar_.reserve(insts.size() * 4 * sizeof(float));
        o_nnz_ = ar_.reserve(insts.size() * sizeof(unsigned long long));
        o_inexact_ = ar_.reserve(insts.size() * sizeof(int));
        o_hist_ = ar_.reserve(UBQP_HIST_BINS * sizeof(int64_t));
        o_active_ = ar_.reserve(sizeof(int32_t));
        o_bytes_ = ar_.reserve(sizeof(unsigned long long));

        // lanes: rows per phase-A item for the GEMV path
        int64_t total_rows = 0;
        for (const LaneIn& l : lanes) total_rows += insts[l.inst].n;
        // rows per phase-A item: enough items to fill the GPU with all lanes active, and at
        // most 32 rows.  Longer items spread each item's fixed costs (its barriers, epilogue
        // and partial) over more bytes; measured on the 40-lane sweep: 16 rows 69.7 % of the
        // HBM peak, 32 rows 75.2 %, 64 rows 57.8 % (too few items once few lanes are left)
        int target_items = 8 * num_sms_;
        int rb = 8;
        while (rb < 32 && total_rows / rb > target_items) rb *= 2;
        if (o_.rows_per_item > 0) rb = o_.rows_per_item;
        if (sym_) rb = kSymT;   // the second stage works on whole tile rows
        // sliced storage: items of whole 32-row slices (32, 64, 128 or 256 rows); one slice per
        // item unless the caller asked for another of these (measured on the 40-lane sweep:
        // 32 rows 13.7 s per step, 64 rows 13.9 s, 128 rows 15.5 s: the eight warps of a slice
        // keep more loads in flight than two)
        if (sparse_) rb = (o_.rows_per_item == 64 || o_.rows_per_item == 128 || o_.rows_per_item == 256) ? o_.rows_per_item : 32;
        // FP32 lanes on the single-lane persistent kernel (a cooperative launch in which each lane
        // runs on its own group of CTAs): one lane whenever its vectors fit in shared memory; several
        // lanes on the sliced storage when every lane gets a group of CTAs that owns at most
        // kSoloMaxSl slices each, all groups resident at once; or when the caller asks for it
        const bool solo_fit = !tc && !sym_ && 2 * (size_t)max_ld * sizeof(float) <= 200 * 1024;
        const bool solo_auto = o_.gemv_kernel == 0 && o_.profile_kernels < 2;
        if (!tc && o_.gemv_kernel == 3 && !solo_fit) {
            set_error("the single-lane kernel keeps two vectors of ld floats in shared memory: ld <= 25600");
            return UBQP_ENOTSUP;
        }
        solo_ = solo_fit && (o_.gemv_kernel == 3 || (solo_auto && (lanes.size() == 1 || sparse_)));
        if (solo_ && lanes.size() == 1 && sparse_) {
            // one CTA per 32-row slice (one CTA for up to 256 rows), unless the caller chose
            const int n0 = (int)insts[lanes[0].inst].n;
            if (o_.rows_per_item != 64 && o_.rows_per_item != 128 && o_.rows_per_item != 256 && o_.rows_per_item != 32)
            {
                rb = 32;   // one slice per CTA; up to 256 rows: one CTA of 32, 64, 128 or 256 rows
                if (n0 <= 256)
                    while (rb < n0) rb *= 2;
            }
            solo_nblk_ = (n0 + rb - 1) / rb;
            solo_grid_ = std::min(solo_nblk_, num_sms_);
        } else if (solo_ && lanes.size() == 1) {
            solo_shape((int)insts[lanes[0].inst].n, o_.rows_per_item, num_sms_, &solo_grid_, &rb, &solo_nblk_);
        }
        if (solo_ && lanes.size() > 1) {
            solo_nb_.assign(lanes.size(), 0);
            std::vector<int> ids(lanes.size());
            for (size_t l = 0; l < lanes.size(); ++l) {
                solo_nb_[l] = (int)((insts[lanes[l].inst].n + rb - 1) / rb);
                ids[l] = (int)l;
            }
            const bool ok = plan_solo_groups(ids, max_ld, o_.gemv_kernel == 3);
            if (!ok && o_.gemv_kernel == 3) {
                set_error("the lanes do not fit the single-lane kernel");
                return UBQP_ENOTSUP;
            }
            solo_ = ok;
        } else if (solo_) {
            solo_glanes_.assign(1, 0);
            solo_gfirst_ = {0, 1};
            solo_gcta_ = {0, solo_grid_};
            solo_one_ok_ = solo_grid_ == 1 && 6 * (size_t)max_ld * sizeof(float) <= 200 * 1024;
        }
        rows_per_item_ = rb;

        lanes_.assign(lanes.size(), LaneDev());
        lane_init_.resize(lanes.size());
        o_vec_.resize(lanes.size());
        o_bx_.resize(lanes.size());
        o_part_.resize(lanes.size());
        o_trace_x_.assign(lanes.size(), 0);
        o_trace_a_.assign(lanes.size(), 0);
        o_x0_.assign(lanes.size(), SIZE_MAX);
        o_p0_.assign(lanes.size(), SIZE_MAX);
        sym_host_.assign(sym_ ? lanes.size() : 0, SymLane());
        o_pbuf_.assign(lanes.size(), 0);
        int64_t nitems = 0;
        lane_inst_.assign(lanes.size(), 0);
        for (size_t l = 0; l < lanes.size(); ++l) {
            const LaneIn& in = lanes[l];
            InstDev& I = inst_[in.inst];
            lane_inst_[l] = in.inst;
            if (I.lane0 < 0) I.lane0 = (int)l;
            I.nl += 1;
            LaneDev& L = lanes_[l];
            L.n = (int)I.n;
            L.ld = I.ld;
            L.mode = tc ? MODE_TC : MODE_GEMV;
            L.nblk = tc ? (int)(I.ld / 128) : (int)((I.n + rb - 1) / rb);
            L.method = o_.method;
            L.stop_after = in.stop_after;
            L.restart = in.restart;
            L.trace_len = in.trace_len;
            if (sym_) {
                sym_host_[l].nb = I.nb;
                sym_host_[l].ntiles = I.nb * (I.nb + 1) / 2;
                sym_host_[l].ngroups = (sym_host_[l].ntiles + kSymGroup - 1) / kSymGroup;
                o_pbuf_[l] = ar_.reserve((size_t)I.nb * I.ld * 4);
            }
            if (!tc) nitems += sym_ ? sym_slots(sym_host_[l]) : L.nblk;
            o_vec_[l] = ar_.reserve((size_t)NVEC * I.ld * 4);
            o_bx_[l] = ar_.reserve((size_t)I.ld);
            // the single-lane kernel's one-barrier steps alternate between two sets of records
            o_part_[l] = ar_.reserve((size_t)(solo_ ? 2 : 1) * L.nblk * sizeof(Partial));
            if (in.trace_len > 0) {
                o_trace_x_[l] = ar_.reserve((size_t)in.trace_len * I.n * 4);
                o_trace_a_[l] = ar_.reserve((size_t)in.trace_len * 4);
            }
            if (in.x0) o_x0_[l] = is_device_ptr(in.x0) ? SIZE_MAX - 1 : ar_.reserve((size_t)I.n * 8);
            if (in.p0) o_p0_[l] = is_device_ptr(in.p0) ? SIZE_MAX - 1 : ar_.reserve((size_t)I.n * 8);
        }
        if (tc) {
            for (InstDev& I : inst_) {
                const int rpad = (int)round_up((size_t)I.nl, 16);
                I.bn = rpad < kTcMaxBn ? rpad : kTcMaxBn;
                I.n_tiles = (rpad + I.bn - 1) / I.bn;
                I.rows_b = I.n_tiles * I.bn;
                I.o_Uhi = ar_.reserve((size_t)I.rows_b * I.ld * 2);
                I.o_Ulo = o_.precision == UBQP_BF16X2_TC ? ar_.reserve((size_t)I.rows_b * I.ld * 2) : 0;
                I.ntact = ntact_total_;
                ntact_total_ += (size_t)I.n_tiles;
            }
            o_ntact_ = ar_.reserve(ntact_total_ * sizeof(int32_t));
            o_tcinst_ = ar_.reserve(inst_.size() * sizeof(TcInst));
            o_tcerr_ = ar_.reserve(sizeof(int32_t));
        }
        o_flops_ = ar_.reserve(sizeof(unsigned long long));
        o_states_ = ar_.reserve(lanes.size() * sizeof(LaneState));
        o_counters_ = ar_.reserve(lanes.size() * sizeof(unsigned int));
        o_symctr_ = sym_ ? ar_.reserve(lanes.size() * sizeof(unsigned int)) : 0;
        o_symlanes_ = sym_ ? ar_.reserve(lanes.size() * sizeof(SymLane)) : 0;
        o_queue_ = ar_.reserve(2 * sizeof(int32_t));
        // single-lane kernel: err, active_after, then one barrier of kSoloBarStride words per group,
        // then the group tables
        // (room for the largest plan: a group per lane, or one per resident CTA)
        const size_t nsg = solo_ ? (size_t)std::max<int64_t>((int64_t)lanes.size(), solo_capc_) : 1;
        o_solo_ = ar_.reserve((4 + nsg * kSoloBarStride) * sizeof(int32_t));
        solo_gmax_ = nsg;
        solo_nl_ = (int)lanes.size();
        o_sologrp_ = solo_ ? ar_.reserve((lanes.size() + 2 * (nsg + 1)) * sizeof(int32_t)) : 0;
        o_lanes_ = ar_.reserve(lanes.size() * sizeof(LaneDev));
        o_linit_ = ar_.reserve(lanes.size() * sizeof(LaneInit));
        o_items_ = ar_.reserve((size_t)std::max<int64_t>(nitems, 1) * sizeof(int2));
        o_final_lane0_ = ar_.reserve(insts.size() * 4);
        o_final_nl_ = ar_.reserve(insts.size() * 4);
        o_final_obj_ = ar_.reserve(insts.size() * 8);
        o_final_best_ = ar_.reserve(insts.size() * 4);
        o_final_xptr_ = ar_.reserve(insts.size() * sizeof(void*));
        o_final_xbuf_ = 0;
        size_t xbuf = 0;
        for (InstDev& I : inst_) xbuf += round_up((size_t)I.n, 256);
        o_final_xbuf_ = ar_.reserve(xbuf);
        nitems_ = (int)nitems;
        if (!tc && nitems > 0 && !solo_) {
            // scheduler of the FP32 lanes: the persistent lane loop, unless the lock-step
            // tick kernel is asked for (or the per-tick timeline, which needs one launch per
            // tick); ring entries hold lane and block indices in 16 bits each
            int max_nblk = 0;
            for (const LaneDev& L : lanes_) max_nblk = std::max(max_nblk, L.nblk);
            const bool fits = lanes.size() < 0xFFFEu && max_nblk <= 0xFFFF;
            if (o_.gemv_kernel == 2 && !fits) {
                set_error("the lane loop takes at most 65533 lanes of at most 65535 row blocks");
                return UBQP_ENOTSUP;
            }
            // automatic choice: the loop pays off once several lanes can overlap one another's
            // update latency; one to three lanes step faster in lock-step
            loop_ = sym_ || (fits && (o_.gemv_kernel == 2 ||
                                      (o_.gemv_kernel == 0 && o_.profile_kernels < 2 && lanes.size() >= 4)));
            if (loop_) {
                UBQP_CK(prepare_lane_loop(max_ld));
                loop_grid_ = lane_loop_grid(max_ld);
                loop_cap_ = 1024;
                while (loop_cap_ < 2 * ((uint64_t)nitems + (uint64_t)loop_grid_)) loop_cap_ *= 2;
                loop_budget_ = probe_ticks_ > 0 ? probe_ticks_ : (o_.lane_budget > 0 ? o_.lane_budget : 1024);
                o_ring_ = ar_.reserve(loop_cap_ * sizeof(unsigned long long));
                o_ht_ = ar_.reserve(2 * sizeof(unsigned long long));
                o_loopctr_ = ar_.reserve(3 * sizeof(int32_t));
                o_budget_ = ar_.reserve(lanes.size() * sizeof(int32_t));
            }
        }
        rc = ar_.commit();
        if (rc) return rc;
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_hist_), 0, UBQP_HIST_BINS * sizeof(int64_t), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_bytes_), 0, sizeof(unsigned long long), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_flops_), 0, sizeof(unsigned long long), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_counters_), 0, lanes.size() * sizeof(unsigned int), stream_));
        if (sym_) UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_symctr_), 0, lanes.size() * sizeof(unsigned int), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_queue_), 0, 2 * sizeof(int32_t), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_solo_), 0, (4 + nsg * kSoloBarStride) * sizeof(int32_t), stream_));
        if (solo_) UBQP_CK(upload_solo_plan());
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_valid_), 0, insts.size() * 4 * sizeof(float), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_nnz_), 0, insts.size() * sizeof(unsigned long long), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_scal_), 0, insts.size() * 4 * sizeof(float), stream_));
        UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_inexact_), 0, insts.size() * sizeof(int), stream_));

        // ---- stage inputs
        for (size_t t = 0; t < insts.size(); ++t) {
            const InstIn& in = insts[t];
            InstDev& I = inst_[t];
            const size_t n = (size_t)in.n;
            I.Q = in.Q;
            I.b = in.b;
            I.mu = in.mu;
            I.starts = in.starts;
            if (I.Q_host) {
                UBQP_CK(cudaMemcpyAsync(ar_.at<double>(I.o_Q), in.Q, n * n * 8, cudaMemcpyHostToDevice, stream_));
                I.Q = ar_.at<double>(I.o_Q);
            }
            if (I.b_host) {
                UBQP_CK(cudaMemcpyAsync(ar_.at<double>(I.o_b), in.b, n * 8, cudaMemcpyHostToDevice, stream_));
                I.b = ar_.at<double>(I.o_b);
            }
            if (I.mu_host) {
                UBQP_CK(cudaMemcpyAsync(ar_.at<double>(I.o_mu), in.mu, n * n * 8, cudaMemcpyHostToDevice, stream_));
                I.mu = ar_.at<double>(I.o_mu);
            }
        }
        // ---- validate (Q symmetric, finite): one launch over every row of every instance
        const int ninst = (int)insts.size();
        std::vector<int64_t> row0(ninst + 1, 0);
        for (int t = 0; t < ninst; ++t) row0[t + 1] = row0[t] + inst_[t].n;
        {
            std::vector<ValArgs> va(ninst);
            for (int t = 0; t < ninst; ++t) {
                va[t].Q = inst_[t].Q;
                va[t].b = inst_[t].b;
                va[t].n = (int)inst_[t].n;
                va[t].pad_ = 0;
                va[t].out = ar_.at<float>(o_valid_) + 4 * t;
                va[t].nnz = ar_.at<unsigned long long>(o_nnz_) + t;
            }
            UBQP_CK(cudaMemcpyAsync(ar_.at<int64_t>(o_row0_), row0.data(), row0.size() * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, stream_));
            UBQP_CK(cudaMemcpyAsync(ar_.at<ValArgs>(o_valargs_), va.data(), va.size() * sizeof(ValArgs),
                                    cudaMemcpyHostToDevice, stream_));
            UBQP_CK(launch_validate(ar_.at<ValArgs>(o_valargs_), ar_.at<int64_t>(o_row0_), ninst, row0[ninst], stream_));
            launches_ += 1;
        }
        std::vector<float> val(insts.size() * 4);
        UBQP_CK(cudaMemcpyAsync(val.data(), ar_.at<float>(o_valid_), val.size() * 4, cudaMemcpyDeviceToHost, stream_));
        nnz_host_.assign(insts.size(), 0);
        UBQP_CK(cudaMemcpyAsync(nnz_host_.data(), ar_.at<unsigned long long>(o_nnz_),
                                insts.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        for (size_t t = 0; t < insts.size(); ++t) {
            if (val[4 * t + 2] != 0.f) { set_error("instance %zu: Q or b holds NaN/Inf", t); return UBQP_ENONFINITE; }
            if (val[4 * t + 0] > 1e-12f * std::max(val[4 * t + 3], 1e-30f)) {
                set_error("instance %zu: Q is not symmetric (max |Q_ij - Q_ji| = %g)", t, val[4 * t + 0]);
                return UBQP_ENOTSYM;
            }
        }
        // ---- reformulate (Sec. 3.5): one launch over every row of every instance
        std::vector<RefArgs> refs(insts.size());
        for (size_t t = 0; t < insts.size(); ++t) {
            const InstIn& in = insts[t];
            InstDev& I = inst_[t];
            RefArgs& a = refs[t];
            memset(&a, 0, sizeof(a));
            a.n = (int)I.n;
            a.ld = I.ld;
            a.inst = (int)t;
            a.diag_only_mu = tc ? 1 : 0;
            a.Q = I.Q;
            a.b = I.b;
            a.mu = in.reformulated ? nullptr : I.mu;
            double offmax = val[4 * t + 1];
            a.sigma = (in.reformulated || I.mu) ? 0.0 : o_.sigma_rel * (offmax > 0 ? offmax : 1.0);
            a.margin = in.reformulated ? 0.0 : o_.gamma_margin;
            a.seed = o_.seed;
            a.Qoff = tc ? nullptr : ar_.at<float>(I.o_Qoff);
            a.Qbf = tc ? ar_.at<__nv_bfloat16>(I.o_Qbf) : nullptr;
            a.Qeval = tc ? nullptr : ar_.at<float2>(I.o_Qeval);
            a.d = ar_.at<float>(I.o_d);
            a.bprime = ar_.at<float>(I.o_bp);
            a.oabs = ar_.at<float>(I.o_oabs);
            a.rabs = ar_.at<float>(I.o_rabs);
            a.tsum = ar_.at<float>(I.o_tsum);
            a.borig = ar_.at<double>(I.o_borig);
            a.qdb = ar_.at<double>(I.o_qdb);
            a.gamma = ar_.at<double>(I.o_gamma);
            a.scal = ar_.at<float>(o_scal_) + 4 * t;
            a.inexact = ar_.at<int>(o_inexact_) + t;
            a.no_gamma = in.reformulated ? 1 : 0;  // Q', b' given: no shift
            if (tc && I.nl > 0 && a.Qbf) {
                // zero the padded rows of the BF16 matrix (rows n..ld-1)
                if ((size_t)I.ld > (size_t)I.n)
                    // rows n..ld-1 all lie in the last M tile: clear its tiles, the reformulation
                    // then writes rows < n over them
                    UBQP_CK(cudaMemsetAsync(a.Qbf + qbf_index((size_t)(I.ld - 128), 0, (size_t)I.ld), 0,
                                            (size_t)128 * I.ld * 2, stream_));
            }
        }
        UBQP_CK(cudaMemcpyAsync(ar_.at<RefArgs>(o_refargs_), refs.data(), refs.size() * sizeof(RefArgs),
                                cudaMemcpyHostToDevice, stream_));
        UBQP_CK(launch_reformulate(ar_.at<RefArgs>(o_refargs_), ar_.at<int64_t>(o_row0_), ninst, row0[ninst], stream_));
        launches_ += 2;
        if (sym_)
            for (InstDev& I : inst_) {
                if (I.nl == 0) continue;
                UBQP_CK(launch_pack_sym(ar_.at<float>(I.o_Qoff), (int)I.n, I.ld, ar_.at<float>(I.o_Qsym), stream_));
                launches_ += 1;
            }
        if (sparse_) {
            int rc2 = build_sliced();
            if (rc2) return rc2;
        }
        std::vector<float> scal(insts.size() * 4);
        UBQP_CK(cudaMemcpyAsync(scal.data(), ar_.at<float>(o_scal_), scal.size() * 4, cudaMemcpyDeviceToHost, stream_));
        std::vector<int> inexact(insts.size());
        UBQP_CK(cudaMemcpyAsync(inexact.data(), ar_.at<int>(o_inexact_), inexact.size() * sizeof(int),
                                cudaMemcpyDeviceToHost, stream_));
        // ---- stage lane-specific inputs
        for (size_t l = 0; l < lanes.size(); ++l) {
            const LaneIn& in = lanes[l];
            const size_t n = (size_t)inst_[in.inst].n;
            const double* x0 = in.x0;
            const double* p0 = in.p0;
            if (in.x0 && o_x0_[l] != SIZE_MAX - 1) {
                UBQP_CK(cudaMemcpyAsync(ar_.at<double>(o_x0_[l]), in.x0, n * 8, cudaMemcpyHostToDevice, stream_));
                x0 = ar_.at<double>(o_x0_[l]);
            }
            if (in.p0 && o_p0_[l] != SIZE_MAX - 1) {
                UBQP_CK(cudaMemcpyAsync(ar_.at<double>(o_p0_[l]), in.p0, n * 8, cudaMemcpyHostToDevice, stream_));
                p0 = ar_.at<double>(o_p0_[l]);
            }
            lane_init_[l].phase = in.phase;
            lane_init_[l].start_kind = in.start_kind;
            lane_init_[l].inst = in.inst;
            lane_init_[l].restart = in.restart;
            lane_init_[l].x0 = x0;
            lane_init_[l].p0 = p0;
        }
        UBQP_CK(cudaStreamSynchronize(stream_));
        inexact_ = false;
        for (int v : inexact) inexact_ |= (v != 0);
        if (tc && inexact_) {
            set_error("tensor-core precision needs every off-diagonal entry exactly representable in BF16; "
                      "use UBQP_FP32 for this data");
            return UBQP_ENOTSUP;
        }
        // ---- lane descriptors
        std::vector<int2> items;
        items.reserve((size_t)nitems);
        for (size_t l = 0; l < lanes.size(); ++l) {
            const LaneIn& in = lanes[l];
            InstDev& I = inst_[in.inst];
            LaneDev& L = lanes_[l];
            L.Qoff = tc ? nullptr : ar_.at<float>(I.o_Qoff);
            if (sparse_ && I.nl > 0) {
                L.spv = sp_ar_.at<float>(I.o_spv);
                L.spc = sp_ar_.at<uint16_t>(I.o_spc);
                L.spo = sp_ar_.at<int64_t>(I.o_spo);
                L.spwps = 256 / rows_per_item_;   // 256 threads per GEMV CTA
            }
            L.Qeval = tc ? nullptr : ar_.at<float2>(I.o_Qeval);
            L.d = ar_.at<float>(I.o_d);
            L.bprime = ar_.at<float>(I.o_bp);
            L.oabs = ar_.at<float>(I.o_oabs);
            L.rabs = ar_.at<float>(I.o_rabs);
            L.tsum = ar_.at<float>(I.o_tsum);
            L.borig = ar_.at<double>(I.o_borig);
            L.qdb = ar_.at<double>(I.o_qdb);
            L.vec = ar_.at<float>(o_vec_[l]);
            L.best_x = ar_.at<uint8_t>(o_bx_[l]);
            L.part = ar_.at<Partial>(o_part_[l]);
            L.st = ar_.at<LaneState>(o_states_) + l;
            L.counter = ar_.at<unsigned int>(o_counters_) + l;
            if (sym_) {
                SymLane& S = sym_host_[l];
                S.Qsym = ar_.at<float>(I.o_Qsym);
                S.pbuf = ar_.at<float>(o_pbuf_[l]);
                S.counter = ar_.at<unsigned int>(o_symctr_) + l;
            }
            if (tc) {
                L.u_hi = ar_.at<__nv_bfloat16>(I.o_Uhi) + (size_t)in.restart * I.ld;
                L.u_lo = I.o_Ulo ? ar_.at<__nv_bfloat16>(I.o_Ulo) + (size_t)in.restart * I.ld : nullptr;
                L.nt_active = ar_.at<int32_t>(o_ntact_) + I.ntact + in.restart / I.bn;
            }
            L.trace_x = in.trace_len > 0 ? ar_.at<float>(o_trace_x_[l]) : nullptr;
            L.trace_alpha = in.trace_len > 0 ? ar_.at<float>(o_trace_a_[l]) : nullptr;
            L.qmax_off = scal[4 * in.inst + 0];
            L.rabs_max = scal[4 * in.inst + 1];
        }
        if (!tc) {   // largest lanes first in the GEMV work queue
            std::vector<int> order(lanes.size());
            for (size_t l = 0; l < lanes.size(); ++l) order[l] = (int)l;
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lanes_[a].n > lanes_[b].n; });
            for (int l : order)
                for (int b = 0; b < (sym_ ? sym_slots(sym_host_[l]) : lanes_[l].nblk); ++b) items.push_back(make_int2(l, b));
        }
        if (sym_)
            UBQP_CK(cudaMemcpyAsync(ar_.at<SymLane>(o_symlanes_), sym_host_.data(), sym_host_.size() * sizeof(SymLane),
                                    cudaMemcpyHostToDevice, stream_));
        UBQP_CK(cudaMemcpyAsync(ar_.at<LaneDev>(o_lanes_), lanes_.data(), lanes_.size() * sizeof(LaneDev),
                                cudaMemcpyHostToDevice, stream_));
        UBQP_CK(cudaMemcpyAsync(ar_.at<LaneInit>(o_linit_), lane_init_.data(), lane_init_.size() * sizeof(LaneInit),
                                cudaMemcpyHostToDevice, stream_));
        if (!items.empty())
            UBQP_CK(cudaMemcpyAsync(ar_.at<int2>(o_items_), items.data(), items.size() * sizeof(int2),
                                    cudaMemcpyHostToDevice, stream_));
        if (loop_) {
            UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_ring_), 0, loop_cap_ * sizeof(unsigned long long), stream_));
            UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_ht_), 0, 2 * sizeof(unsigned long long), stream_));
            UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_loopctr_), 0, 3 * sizeof(int32_t), stream_));
        }
        if (tc) {
            for (InstDev& I : inst_) {
                UBQP_CK(cudaMemsetAsync(ar_.at<char>(I.o_Uhi), 0, (size_t)I.rows_b * I.ld * 2, stream_));
                if (I.o_Ulo) UBQP_CK(cudaMemsetAsync(ar_.at<char>(I.o_Ulo), 0, (size_t)I.rows_b * I.ld * 2, stream_));
            }
            UBQP_CK(cudaMemsetAsync(ar_.at<char>(o_tcerr_), 0, sizeof(int32_t), stream_));
            // tile table with the TMA descriptors of every instance, largest instances first:
            // CTAs take tiles at a fixed stride, and this order deals every CTA a similar mix of
            // long and short tiles (the table order does not change any result)
            std::vector<TcInst> ti(inst_.size());
            ntact_host_.assign(ntact_total_, 0);
            std::vector<size_t> by_size(inst_.size());
            for (size_t t = 0; t < inst_.size(); ++t) by_size[t] = t;
            std::stable_sort(by_size.begin(), by_size.end(),
                             [&](size_t a, size_t b) { return inst_[a].ld > inst_[b].ld; });
            int cl = 0, kb_min = 1 << 30;
            max_bn_ = 16;
            for (size_t q = 0; q < inst_.size(); ++q) {
                const size_t t = by_size[q];
                InstDev& I = inst_[t];
                TcInst& h = ti[q];
                memset(&h, 0, sizeof(h));
                const void* ub = ar_.at<char>(I.o_Uhi);
                const void* lb = I.o_Ulo ? (const void*)ar_.at<char>(I.o_Ulo) : ub;
                if (tc_encode_map(&h.tmA, ar_.at<char>(I.o_Qbf), (int64_t)I.ld * I.ld / 64, 64, 128) != CUDA_SUCCESS ||
                    tc_encode_map(&h.tmBhi, ub, I.rows_b, I.ld, I.bn) != CUDA_SUCCESS ||
                    tc_encode_map(&h.tmBlo, lb, I.rows_b, I.ld, I.bn) != CUDA_SUCCESS) {
                    set_error("cuTensorMapEncodeTiled failed for instance %zu", t);
                    return UBQP_ECUDA;
                }
                h.n = (int)I.n;
                h.ld = I.ld;
                h.R = I.nl;
                h.lane0 = I.lane0;
                h.m_tiles = I.ld / 128;
                h.n_tiles = I.n_tiles;
                h.bn = I.bn;
                h.two_terms = I.o_Ulo ? 1 : 0;
                h.cluster0 = cl;
                h.nt_active = ar_.at<int32_t>(o_ntact_) + I.ntact;
                for (int q = 0; q < I.n_tiles; ++q) ntact_host_[I.ntact + q] = std::min(I.bn, I.nl - q * I.bn);
                cl += h.m_tiles * h.n_tiles;
                kb_min = std::min(kb_min, I.ld / 64);
                max_bn_ = std::max(max_bn_, I.bn);
            }
            tc_tiles_ = cl;
            UBQP_CK(cudaMemcpyAsync(ar_.at<TcInst>(o_tcinst_), ti.data(), ti.size() * sizeof(TcInst),
                                    cudaMemcpyHostToDevice, stream_));
            UBQP_CK(cudaMemcpyAsync(ar_.at<int32_t>(o_ntact_), ntact_host_.data(), ntact_total_ * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, stream_));
            const bool two = o_.precision == UBQP_BF16X2_TC;
            tc_stages_ = tc_pick_stages(max_bn_, two);
            tc_S_ = o_.tc_cluster > 0 ? o_.tc_cluster
                                      : tc_pick_cluster(tc_tiles_, kb_min, max_bn_, two, tc_stages_, num_sms_);
            // enough tiles for the whole GPU without splitting K: the persistent kernel, which
            // overlaps each tile's epilogue with the next tile's contraction
            const int tcp_stages = tcp_pick_stages(max_bn_, two);
            tcp_ = tc_S_ == 1 && tcp_stages >= 2 && tc_tiles_ >= num_sms_;
            if (tcp_) tc_stages_ = tcp_stages;
        }
        LaneInitArgs lia;
        lia.lanes = ar_.at<LaneDev>(o_lanes_);
        lia.init = ar_.at<LaneInit>(o_linit_);
        lia.seed = o_.seed;
        UBQP_CK(launch_lane_init(lia, (int)lanes.size(), stream_));
        launches_ += 1;
        // host copies of the vectors are no longer needed; keep them for stats
        nlanes_ = (int)lanes.size();
        return UBQP_OK;
    }

    // Tensor-core launch form by measurement (tc_cluster = 0): every feasible split-K cluster
    // size S (each CTA keeps >= 2 k-blocks, at least one cluster fits) and, when its ring
    // fits, the persistent many-tile kernel each run one warm-up and three timed launches of
    // the contraction alone on this call's operands (raw output into a scratch buffer; no lane
    // state is read or written); the fastest (shortest of its three) is kept.
    int tune_tc_form()
    {
        if (!tc_ || tc_tiles_ == 0 || o_.tc_cluster > 0) return UBQP_OK;
        const bool two = o_.precision == UBQP_BF16X2_TC;
        int dev = 0, major = 0, minor = 0;
        UBQP_CK(cudaGetDevice(&dev));
        UBQP_CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
        UBQP_CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
        int kb_min = 1 << 30;
        size_t raw_elems = 1;
        for (const InstDev& I : inst_) {
            kb_min = std::min(kb_min, I.ld / 64);
            raw_elems = std::max(raw_elems, (size_t)I.nl * (size_t)I.ld);
        }
        char key[160];
        snprintf(key, sizeof(key), "sm%d%d:sms%d:tiles%d:kb%d:bn%d:terms%d:inst%zu:ld%d", major, minor, num_sms_,
                 tc_tiles_, kb_min, max_bn_, two ? 2 : 1, inst_.size(), max_ld_);
        const char* path = getenv("UBQP_TUNE_CACHE");
        int choice = -1;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            tune_load_file_locked(path);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) choice = it->second;
        }
        const int tcp_stages = tcp_pick_stages(max_bn_, two);
        if (choice >= 0 && choice <= 8 && !(choice == 0 && tcp_stages < 2)) {
            cluster_tuned_ = 2;
        } else {
            float* raw = nullptr;
            UBQP_CK(cudaMallocAsync((void**)&raw, raw_elems * sizeof(float), stream_));
            AsyncTemp guard;
            guard.hold(raw, stream_);
            TcArgs a;
            memset(&a, 0, sizeof(a));
            a.inst = ar_.at<TcInst>(o_tcinst_);
            a.ninst = (int)inst_.size();
            a.max_bn = max_bn_;
            a.two_any = two ? 1 : 0;
            a.lanes = ar_.at<LaneDev>(o_lanes_);
            a.raw = raw;
            a.err = ar_.at<int32_t>(o_tcerr_);
            a.P = make_params(o_, nullptr);
            cudaEvent_t e0, e1;
            UBQP_CK(cudaEventCreate(&e0));
            UBQP_CK(cudaEventCreate(&e1));
            float best = INFINITY;
            for (int S = 0; S <= 8; ++S) {
                cudaError_t le = cudaSuccess;
                if (S == 0) {
                    if (tcp_stages < 2) continue;
                    a.stages = tcp_stages;
                    a.tmem_cols = tcp_tmem_cols(two);
                } else {
                    if (S > 1 && kb_min / S < 2) break;
                    a.stages = tc_pick_stages(max_bn_, two);
                    a.tmem_cols = tc_tmem_cols(max_bn_, two);
                    if (tc_max_active_clusters(max_bn_, two, a.stages, S) < 1) continue;
                }
                const int grid = S == 0 ? tcp_grid(a, tc_tiles_) : 0;
                float t = INFINITY;
                for (int rep = 0; rep < 4 && le == cudaSuccess; ++rep) {
                    le = cudaEventRecord(e0, stream_);
                    if (le == cudaSuccess)
                        le = S == 0 ? tcp_launch(a, tc_tiles_, grid, stream_) : tc_launch(a, tc_tiles_, S, stream_);
                    if (le == cudaSuccess) le = cudaEventRecord(e1, stream_);
                    if (le == cudaSuccess) le = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (le == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                        t = std::min(t, ms * 1e3f);
                }
                if (le != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    set_error("tensor-core form probe (S = %d) failed: %s", S, cudaGetErrorString(le));
                    return UBQP_ECUDA;
                }
                cluster_probe_us_[S] = t;
                if (t < best) {
                    best = t;
                    choice = S;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            int32_t err = 0;
            UBQP_CK(cudaMemcpy(&err, a.err, sizeof(err), cudaMemcpyDeviceToHost));
            if (err) {
                set_error("a bounded wait in the tensor-core kernel ran out while tuning its launch form");
                return UBQP_ETIMEOUT;
            }
            guard.release();
            UBQP_CK(cudaFreeAsync(raw, stream_));
            if (choice < 0) choice = 1;
            cluster_tuned_ = 1;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = choice;
            tune_save_file_locked(path);
        }
        if (choice == 0) {
            tc_S_ = 1;
            tcp_ = true;
            tc_stages_ = tcp_stages;
        } else {
            tc_S_ = choice;
            tcp_ = false;
            tc_stages_ = tc_pick_stages(max_bn_, two);
        }
        return UBQP_OK;
    }

    int run()
    {
        if (loop_) return run_loop();
        if (solo_) return run_solo();
        {
            const int rc = tune_tc_form();
            if (rc) return rc;
        }
        TickArgs ta;
        ta.lanes = ar_.at<LaneDev>(o_lanes_);
        ta.items = ar_.at<int2>(o_items_);
        ta.nitems = nitems_;
        ta.rows_per_item = rows_per_item_;
        ta.nlanes = nlanes_;
        ta.max_ld = max_ld_;
        ta.fused = 0;
        ta.active_count = nullptr;
        ta.work = ar_.at<int32_t>(o_queue_);
        ta.done = ar_.at<int32_t>(o_queue_) + 1;
        ta.grid = 0;
        ta.P = make_params(o_, ar_.at<int64_t>(o_hist_));
        const bool prof = o_.profile_kernels != 0;
        if (prof) ta.P.bytes = ar_.at<unsigned long long>(o_bytes_);
        int32_t* d_active = ar_.at<int32_t>(o_active_);
        UBQP_CK(cudaMallocHost(&h_active_, sizeof(int32_t)));
        if (!tc_ && nitems_ > 0) {
            UBQP_CK(prepare_phase_a_gemv(max_ld_));
            ta.grid = gemv_grid(max_ld_, nitems_);
        }
        const int T = o_.max_ticks_per_sync;
        const bool has_a = (!tc_ && nitems_ > 0) || (tc_ && tc_tiles_ > 0);
        TcArgs tca;
        memset(&tca, 0, sizeof(tca));
        if (tc_) {
            tca.inst = ar_.at<TcInst>(o_tcinst_);
            tca.ninst = (int)inst_.size();
            tca.stages = tc_stages_;
            tca.tmem_cols = tc_tmem_cols(max_bn_, o_.precision == UBQP_BF16X2_TC);
            tca.max_bn = max_bn_;
            tca.two_any = o_.precision == UBQP_BF16X2_TC ? 1 : 0;
            tca.lanes = ar_.at<LaneDev>(o_lanes_);
            tca.raw = nullptr;
            tca.err = ar_.at<int32_t>(o_tcerr_);
            tca.flops = prof ? ar_.at<unsigned long long>(o_flops_) : nullptr;
            tca.P = ta.P;
            // tc_fuse: the update runs in the contraction's epilogue (lanes of at most 32 M tiles,
            // whose warp-level reduction merges partials in the CTA-level order).  Off by
            // default: every lane of an N tile completes on the same last tile, so one CTA's
            // warps run the updates of the whole N tile one after another (measured on the
            // batched-restart workload: 276 us per step fused, 55 us with the update kernel)
            tca.fuse = (max_ld_ / 128 <= 32 && o_.tc_fuse != 0) ? 1 : 0;
            if (tcp_) {
                tca.tmem_cols = tcp_tmem_cols(o_.precision == UBQP_BF16X2_TC);
                tcp_grid_ = tcp_grid(tca, tc_tiles_);
            }
        }
        const bool timeline = o_.profile_kernels >= 2;
        unsigned long long* d_work_ctr = tc_ ? ar_.at<unsigned long long>(o_flops_) : ar_.at<unsigned long long>(o_bytes_);
        unsigned long long* d_snap = nullptr;
        AsyncTemp snap_guard;
        if (prof && has_a) {
            evA_.resize(2 * T);
            for (auto& e : evA_) UBQP_CK(cudaEventCreate(&e));
            if (timeline) {
                g_tl_ms.clear();
                g_tl_work.clear();
                UBQP_CK(cudaMallocAsync((void**)&d_snap, (size_t)T * sizeof(unsigned long long), stream_));
                snap_guard.hold(d_snap, stream_);
            }
        }

        // GEMV lanes: one fused kernel per tick (the last CTA of each lane updates it);
        // tensor-core lanes: the contraction kernel, whose epilogue warps update the lanes when
        // tca.fuse is set, else followed by the stand-alone update kernel
        const bool fused = has_a && (!tc_ || tca.fuse);
        auto enqueue = [&](int nt) -> cudaError_t {
            for (int t = 0; t < nt; ++t) {
                cudaError_t e = cudaSuccess;
                const bool last = t == nt - 1;
                if (last) {
                    e = cudaMemsetAsync(d_active, 0, sizeof(int32_t), stream_);
                    if (e != cudaSuccess) return e;
                }
                if (prof && has_a) e = cudaEventRecord(evA_[2 * t], stream_);
                if (e != cudaSuccess) return e;
                if (has_a && !tc_) {
                    TickArgs tt = ta;
                    tt.fused = 1;
                    tt.active_count = last ? d_active : nullptr;
                    e = launch_phase_a_gemv_f32(tt, stream_);
                } else if (has_a) {
                    TcArgs tt = tca;
                    tt.active_count = last ? d_active : nullptr;
                    e = tcp_ ? tcp_launch(tt, tc_tiles_, tcp_grid_, stream_) : tc_launch(tt, tc_tiles_, tc_S_, stream_);
                }
                if (e != cudaSuccess) return e;
                if (prof && has_a) e = cudaEventRecord(evA_[2 * t + 1], stream_);
                if (e != cudaSuccess) return e;
                if (d_snap) e = cudaMemcpyAsync(d_snap + t, d_work_ctr, sizeof(unsigned long long),
                                                cudaMemcpyDeviceToDevice, stream_);
                if (e != cudaSuccess) return e;
                if (!fused) {
                    e = launch_phase_b(ta, last ? d_active : nullptr, stream_);
                    if (e != cudaSuccess) return e;
                }
            }
            return cudaMemcpyAsync(h_active_, d_active, sizeof(int32_t), cudaMemcpyDeviceToHost, stream_);
        };
        // capture one batch of T ticks into a graph (profiling launches directly so that
        // the events around every phase-A launch can be timed)
        bool use_graph = !prof;
        if (use_graph && cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t e = enqueue(T);
            cudaError_t e2 = cudaStreamEndCapture(stream_, &graph_);
            if (e != cudaSuccess || e2 != cudaSuccess ||
                cudaGraphInstantiate(&gexec_, graph_, 0) != cudaSuccess) {
                use_graph = false;
                cudaGetLastError();
            }
        } else {
            use_graph = false;
            cudaGetLastError();
        }
        UBQP_CK(cudaEventRecord(ev0_, stream_));
        int64_t ticks = 0;
        const int64_t cap = (int64_t)(o_.jacobi_max_iter + 2) +
                            (int64_t)(o_.max_outer + 1) * (int64_t)(o_.max_inner + o_.lobpcg_max_iter + 8);
        for (;;) {
            if (use_graph) UBQP_CK(cudaGraphLaunch(gexec_, stream_));
            else UBQP_CK(enqueue(T));
            launches_ += (int64_t)T * (fused ? 1 : 2);
            UBQP_CK(cudaStreamSynchronize(stream_));
            ticks += T;
            if (prof && has_a) {
                std::vector<unsigned long long> snap(d_snap ? T : 0);
                if (d_snap)
                    UBQP_CK(cudaMemcpy(snap.data(), d_snap, (size_t)T * sizeof(unsigned long long),
                                       cudaMemcpyDeviceToHost));
                for (int t = 0; t < T; ++t) {
                    float ms = 0.f;
                    UBQP_CK(cudaEventElapsedTime(&ms, evA_[2 * t], evA_[2 * t + 1]));
                    phase_a_ms_ += ms;
                    if (d_snap) {
                        g_tl_ms.push_back(ms);
                        g_tl_work.push_back((int64_t)(snap[t] - tl_prev_));
                        tl_prev_ = snap[t];
                    }
                }
                phase_a_launches_ += T;
            }
            if (tc_) {
                int32_t err = 0;
                UBQP_CK(cudaMemcpy(&err, ar_.at<int32_t>(o_tcerr_), sizeof(err), cudaMemcpyDeviceToHost));
                if (err) {
                    set_error("a bounded wait in the tensor-core kernel ran out");
                    return UBQP_ETIMEOUT;
                }
            }
            if (probe_ticks_ > 0 && ticks >= probe_ticks_) break;
            bool stop = false;
            int rc = check_target(stop);
            if (rc) return rc;
            if (stop) break;
            if (*h_active_ == 0) break;
            if (ticks > cap) {
                set_error("tick cap %lld exceeded", (long long)cap);
                return UBQP_ETIMEOUT;
            }
        }
        UBQP_CK(cudaEventRecord(ev1_, stream_));
        if (d_snap) {
            snap_guard.release();
            UBQP_CK(cudaFreeAsync(d_snap, stream_));
        }
        UBQP_CK(cudaStreamSynchronize(stream_));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0_, ev1_);
        ms_device_ = ms;
        ticks_ = ticks;
        return UBQP_OK;
    }

    // time to the target objective (when one is set): the first host check at which some
    // lane's best exact objective reaches it
    int check_target(bool& stop)
    {
        stop = false;
        if (!std::isfinite(o_.target_objective) || ms_to_target_ >= 0.0) return UBQP_OK;
        std::vector<LaneState> st(nlanes_);
        UBQP_CK(cudaMemcpy(st.data(), ar_.at<LaneState>(o_states_), st.size() * sizeof(LaneState),
                           cudaMemcpyDeviceToHost));
        double best = INFINITY;
        for (const LaneState& x : st) best = std::min(best, x.best_f);
        if (best <= o_.target_objective) {
            UBQP_CK(cudaEventRecord(ev1_, stream_));
            UBQP_CK(cudaEventSynchronize(ev1_));
            float m = 0.f;
            cudaEventElapsedTime(&m, ev0_, ev1_);
            ms_to_target_ = m;
            stop = o_.stop_at_target != 0;
        }
        return UBQP_OK;
    }

    // the sliced storage of every instance with lanes: widths per 32-row slice from the dense
    // FP32 rows, offsets on the host, one allocation, then the packing
    int build_sliced()
    {
        size_t nsl_total = 0;
        std::vector<size_t> sl0(inst_.size());
        for (size_t t = 0; t < inst_.size(); ++t) {
            sl0[t] = nsl_total;
            nsl_total += (size_t)(inst_[t].n + 31) / 32;
        }
        int32_t* dw = nullptr;
        UBQP_CK(cudaMallocAsync((void**)&dw, std::max<size_t>(nsl_total, 1) * sizeof(int32_t), stream_));
        AsyncTemp guard;
        guard.hold(dw, stream_);
        for (size_t t = 0; t < inst_.size(); ++t)
            if (inst_[t].nl > 0)
                UBQP_CK(launch_sell_width(ar_.at<float>(inst_[t].o_Qoff), (int)inst_[t].n, inst_[t].ld, dw + sl0[t], stream_));
        std::vector<int32_t> w(nsl_total, 0);
        UBQP_CK(cudaMemcpyAsync(w.data(), dw, nsl_total * sizeof(int32_t), cudaMemcpyDeviceToHost, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        guard.release();
        UBQP_CK(cudaFreeAsync(dw, stream_));
        std::vector<std::vector<int64_t>> offs(inst_.size());
        for (size_t t = 0; t < inst_.size(); ++t) {
            InstDev& I = inst_[t];
            if (I.nl == 0) continue;
            const size_t ns = (size_t)(I.n + 31) / 32;
            offs[t].assign(ns + 1, 0);
            for (size_t q = 0; q < ns; ++q) offs[t][q + 1] = offs[t][q] + 32 * (int64_t)w[sl0[t] + q];
            const size_t entries = (size_t)offs[t][ns];
            I.o_spv = sp_ar_.reserve(std::max<size_t>(entries, 1) * 4);
            I.o_spc = sp_ar_.reserve(std::max<size_t>(entries, 1) * 2);
            I.o_spo = sp_ar_.reserve((ns + 1) * 8);
            sliced_entries_ += (int64_t)entries;
        }
        int rc = sp_ar_.commit();
        if (rc) return rc;
        for (size_t t = 0; t < inst_.size(); ++t) {
            InstDev& I = inst_[t];
            if (I.nl == 0) continue;
            UBQP_CK(cudaMemcpyAsync(sp_ar_.at<int64_t>(I.o_spo), offs[t].data(), offs[t].size() * 8, cudaMemcpyHostToDevice,
                                    stream_));
            UBQP_CK(launch_sell_pack(ar_.at<float>(I.o_Qoff), (int)I.n, I.ld, sp_ar_.at<int64_t>(I.o_spo),
                                     sp_ar_.at<float>(I.o_spv), sp_ar_.at<uint16_t>(I.o_spc), stream_));
            launches_ += 2;
        }
        UBQP_CK(cudaStreamSynchronize(stream_));   // offsets staged from host vectors
        return UBQP_OK;
    }

    // one FP32 lane on the single-lane persistent kernel: each cooperative launch runs up to
    // lane_budget (1024) steps; the host checks between launches
    int run_solo()
    {
        SoloArgs sa;
        memset(&sa, 0, sizeof(sa));
        sa.lane = ar_.at<LaneDev>(o_lanes_);
        auto set_plan = [&]() {
            const int32_t* tab = ar_.at<int32_t>(o_sologrp_);
            sa.ngroups = (int)solo_gcta_.size() - 1;
            sa.glanes = tab;
            sa.gfirst = tab + solo_nl_;
            sa.gcta = sa.gfirst + solo_gmax_ + 1;
            sa.grid = solo_gcta_.back();
        };
        set_plan();
        sa.rows_per_item = rows_per_item_;
        sa.budget = probe_ticks_ > 0 ? probe_ticks_ : (o_.lane_budget > 0 ? o_.lane_budget : 1024);
        int32_t* ctl = ar_.at<int32_t>(o_solo_);
        sa.err = ctl;
        sa.active_after = ctl + 1;
        sa.bar = reinterpret_cast<unsigned*>(ctl + 4);
        sa.wait_ns = o_.wait_limit_us > 0 ? 1000ull * (unsigned long long)o_.wait_limit_us : 5000000000ull;
        sa.fast = 1;
        sa.one_ok = solo_one_ok_ ? 1 : 0;
        sa.P = make_params(o_, ar_.at<int64_t>(o_hist_));
        const bool prof = o_.profile_kernels != 0;
        if (prof) sa.P.bytes = ar_.at<unsigned long long>(o_bytes_);
        UBQP_CK(prepare_solo(max_ld_, solo_one_ok_));
        UBQP_CK(cudaMallocHost(&h_active_, 2 * sizeof(int32_t)));
        if (prof) {
            evA_.resize(2);
            for (auto& e : evA_) UBQP_CK(cudaEventCreate(&e));
        }
        UBQP_CK(cudaEventRecord(ev0_, stream_));
        const int64_t cap = (int64_t)(o_.jacobi_max_iter + 2) +
                            (int64_t)(o_.max_outer + 1) * (int64_t)(o_.max_inner + o_.lobpcg_max_iter + 8);
        int64_t granted = 0;
        int active_prev = nlanes_;
        for (;;) {
            UBQP_CK(cudaMemsetAsync(sa.active_after, 0, sizeof(int32_t), stream_));
            if (prof) UBQP_CK(cudaEventRecord(evA_[0], stream_));
            UBQP_CK(launch_solo(sa, max_ld_, stream_));
            if (prof) UBQP_CK(cudaEventRecord(evA_[1], stream_));
            UBQP_CK(cudaMemcpyAsync(h_active_, ctl, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream_));
            launches_ += 1;
            granted += sa.budget;
            UBQP_CK(cudaStreamSynchronize(stream_));
            if (prof) {
                float ms = 0.f;
                UBQP_CK(cudaEventElapsedTime(&ms, evA_[0], evA_[1]));
                phase_a_ms_ += ms;
                phase_a_launches_ += 1;
            }
            if (h_active_[0]) {
                set_error("a bounded wait in the single-lane kernel ran out (limit %.0f us)", (double)sa.wait_ns * 1e-3);
                return UBQP_ETIMEOUT;
            }
            if (probe_ticks_ > 0) break;
            bool stop = false;
            int rc = check_target(stop);
            if (rc) return rc;
            if (stop) break;
            if (h_active_[1] == 0) break;
            if (granted > cap * solo_max_lanes_) {
                set_error("step cap %lld exceeded", (long long)cap);
                return UBQP_ETIMEOUT;
            }
            if (nlanes_ > 1 && h_active_[1] < active_prev) {
                // lanes have finished: the CTAs are shared out again over the lanes still running
                // (a lane's arithmetic does not depend on its group, only on its blocks)
                active_prev = h_active_[1];
                std::vector<LaneState> st(nlanes_);
                UBQP_CK(cudaMemcpy(st.data(), ar_.at<LaneState>(o_states_), st.size() * sizeof(LaneState),
                                   cudaMemcpyDeviceToHost));
                std::vector<int> ids;
                for (int l = 0; l < nlanes_; ++l)
                    if (st[l].phase != PH_DONE) ids.push_back(l);
                if (!ids.empty() && plan_solo_groups(ids, max_ld_, true)) {
                    UBQP_CK(upload_solo_plan());
                    set_plan();
                }
            }
        }
        UBQP_CK(cudaEventRecord(ev1_, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0_, ev1_);
        ms_device_ = ms;
        ticks_ = -1;   // filled from the lanes' own step counts
        return UBQP_OK;
    }

    // Groups of CTAs for the given lanes on the single-lane kernel, largest lanes first.  With at
    // most as many lanes as resident CTAs, every lane gets its own group of ceil(nblk / m) CTAs
    // for the smallest m (blocks per CTA) at which all groups are resident together; the
    // automatic choice takes it only for m <= kSoloMaxSl (all of a CTA's slices in one pass).
    // Otherwise (asked for explicitly) one-CTA groups share the lanes, each lane going to the
    // group with the fewest blocks so far.
    bool plan_solo_groups(const std::vector<int>& ids, int max_ld, bool forced)
    {
        const size_t nl = ids.size();
        if (solo_capc_ == 0) {
            solo_one_ok_ = 6 * (size_t)max_ld * sizeof(float) <= 48 * 1024;
            if (prepare_solo(max_ld, solo_one_ok_) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            const int per = solo_ctas_per_sm(max_ld, solo_one_ok_);
            if (per < 1) return false;
            solo_capc_ = (int64_t)per * num_sms_;
        }
        const int64_t capc = solo_capc_;
        std::vector<int> order(ids);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return solo_nb_[a] > solo_nb_[b]; });
        std::vector<int32_t> gl, gf(1, 0), gc(1, 0);
        int max_lanes = 1;
        int maxnb = 0;
        for (int l : ids) maxnb = std::max(maxnb, solo_nb_[l]);
        if ((int64_t)nl <= capc) {
            int m = 1;
            for (; m <= maxnb; ++m) {
                int64_t tot = 0;
                for (int l : ids) tot += (solo_nb_[l] + m - 1) / m;
                if (tot <= capc) break;
            }
            if (!forced && m > kSoloMaxSl) return false;
            for (int l : order) {
                gl.push_back(l);
                gf.push_back((int)gl.size());
                gc.push_back(gc.back() + (solo_nb_[l] + m - 1) / m);
            }
        } else {
            if (!forced) return false;
            const int G = (int)capc;
            std::vector<std::vector<int>> lanes_of(G);
            std::vector<int64_t> load(G, 0);
            for (int l : order) {
                const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                lanes_of[g].push_back(l);
                load[g] += solo_nb_[l];
            }
            for (int g = 0; g < G; ++g) {
                for (int l : lanes_of[g]) gl.push_back(l);
                gf.push_back((int)gl.size());
                gc.push_back(g + 1);
                max_lanes = std::max(max_lanes, (int)lanes_of[g].size());
            }
        }
        solo_glanes_ = gl;
        solo_gfirst_ = gf;
        solo_gcta_ = gc;
        solo_max_lanes_ = std::max(solo_max_lanes_, max_lanes);
        return true;
    }

    // the group tables to the device (glanes, then gfirst and gcta at fixed offsets) and the
    // groups' barrier counters to zero (a new plan regroups the CTAs)
    cudaError_t upload_solo_plan()
    {
        const size_t G1 = solo_gmax_ + 1;
        solo_tab_host_.assign((size_t)solo_nl_ + 2 * G1, 0);
        std::copy(solo_glanes_.begin(), solo_glanes_.end(), solo_tab_host_.begin());
        std::copy(solo_gfirst_.begin(), solo_gfirst_.end(), solo_tab_host_.begin() + solo_nl_);
        std::copy(solo_gcta_.begin(), solo_gcta_.end(), solo_tab_host_.begin() + solo_nl_ + G1);
        cudaError_t e = cudaMemcpyAsync(ar_.at<int32_t>(o_sologrp_), solo_tab_host_.data(),
                                        solo_tab_host_.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream_);
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(ar_.at<int32_t>(o_solo_) + 4, 0, solo_gmax_ * kSoloBarStride * sizeof(int32_t), stream_);
    }

    // FP32 lanes on the persistent lane loop: each launch (seed + loop, one graph) lets
    // every lane take up to loop_budget_ steps; the host checks between launches
    int run_loop()
    {
        LoopArgs la;
        memset(&la, 0, sizeof(la));
        la.lanes = ar_.at<LaneDev>(o_lanes_);
        la.items = ar_.at<int2>(o_items_);
        la.nitems = nitems_;
        la.nlanes = nlanes_;
        la.rows_per_item = rows_per_item_;
        la.max_ld = max_ld_;
        la.budget = loop_budget_;
        la.grid = loop_grid_;
        la.ring = ar_.at<unsigned long long>(o_ring_);
        la.cap = loop_cap_;
        la.head = ar_.at<unsigned long long>(o_ht_);
        la.tail = la.head + 1;
        int32_t* ctr = ar_.at<int32_t>(o_loopctr_);
        la.running = ctr;
        la.active_after = ctr + 1;
        la.err = ctr + 2;
        la.budget_left = ar_.at<int32_t>(o_budget_);
        la.sym = sym_ ? ar_.at<SymLane>(o_symlanes_) : nullptr;
        la.wait_ns = o_.wait_limit_us > 0 ? 1000ull * (unsigned long long)o_.wait_limit_us : 5000000000ull;
        la.P = make_params(o_, ar_.at<int64_t>(o_hist_));
        const bool prof = o_.profile_kernels != 0;
        if (prof) la.P.bytes = ar_.at<unsigned long long>(o_bytes_);
        UBQP_CK(cudaMallocHost(&h_active_, sizeof(int32_t)));
        if (prof) {
            evA_.resize(2);
            for (auto& e : evA_) UBQP_CK(cudaEventCreate(&e));
        }
        auto enqueue = [&]() -> cudaError_t {
            cudaError_t e = prof ? cudaEventRecord(evA_[0], stream_) : cudaSuccess;
            if (e == cudaSuccess) e = launch_lane_loop(la, stream_);
            if (e == cudaSuccess && prof) e = cudaEventRecord(evA_[1], stream_);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_active_, la.active_after, sizeof(int32_t), cudaMemcpyDeviceToHost, stream_);
            return e;
        };
        bool use_graph = !prof;
        if (use_graph && cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t e = enqueue();
            cudaError_t e2 = cudaStreamEndCapture(stream_, &graph_);
            if (e != cudaSuccess || e2 != cudaSuccess || cudaGraphInstantiate(&gexec_, graph_, 0) != cudaSuccess) {
                use_graph = false;
                cudaGetLastError();
            }
        } else {
            use_graph = false;
            cudaGetLastError();
        }
        UBQP_CK(cudaEventRecord(ev0_, stream_));
        const int64_t cap = (int64_t)(o_.jacobi_max_iter + 2) +
                            (int64_t)(o_.max_outer + 1) * (int64_t)(o_.max_inner + o_.lobpcg_max_iter + 8);
        int64_t granted = 0;   // steps granted to each lane so far
        for (;;) {
            if (use_graph) UBQP_CK(cudaGraphLaunch(gexec_, stream_));
            else UBQP_CK(enqueue());
            launches_ += 2;
            granted += loop_budget_;
            UBQP_CK(cudaStreamSynchronize(stream_));
            if (prof) {
                float ms = 0.f;
                UBQP_CK(cudaEventElapsedTime(&ms, evA_[0], evA_[1]));
                phase_a_ms_ += ms;
                phase_a_launches_ += 1;
            }
            int32_t err = 0;
            UBQP_CK(cudaMemcpy(&err, la.err, sizeof(err), cudaMemcpyDeviceToHost));
            if (err) {
                set_error("a bounded wait in the lane loop ran out (limit %.0f us)", (double)la.wait_ns * 1e-3);
                return UBQP_ETIMEOUT;
            }
            if (probe_ticks_ > 0) break;
            bool stop = false;
            int rc = check_target(stop);
            if (rc) return rc;
            if (stop) break;
            if (*h_active_ == 0) break;
            if (granted > cap) {
                set_error("step cap %lld exceeded", (long long)cap);
                return UBQP_ETIMEOUT;
            }
        }
        UBQP_CK(cudaEventRecord(ev1_, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0_, ev1_);
        ms_device_ = ms;
        ticks_ = -1;   // filled from the lanes' own step counts
        return UBQP_OK;
    }

    // best lane per instance; x_out entries are host or device pointers
    int finalize(uint8_t* const* x_out, double* obj_out)
    {
        const size_t ni = inst_.size();
        std::vector<int32_t> l0(ni), nl(ni);
        std::vector<uint8_t*> xd(ni);
        size_t off = 0;
        std::vector<bool> xhost(ni);
        for (size_t t = 0; t < ni; ++t) {
            l0[t] = inst_[t].lane0;
            nl[t] = inst_[t].nl;
            xhost[t] = !is_device_ptr(x_out[t]);
            xd[t] = xhost[t] ? ar_.at<uint8_t>(o_final_xbuf_) + off : x_out[t];
            off += round_up((size_t)inst_[t].n, 256);
        }
        UBQP_CK(cudaMemcpyAsync(ar_.at<int32_t>(o_final_lane0_), l0.data(), ni * 4, cudaMemcpyHostToDevice, stream_));
        UBQP_CK(cudaMemcpyAsync(ar_.at<int32_t>(o_final_nl_), nl.data(), ni * 4, cudaMemcpyHostToDevice, stream_));
        UBQP_CK(cudaMemcpyAsync(ar_.at<uint8_t*>(o_final_xptr_), xd.data(), ni * sizeof(void*), cudaMemcpyHostToDevice,
                                stream_));
        FinalArgs fa;
        fa.lanes = ar_.at<LaneDev>(o_lanes_);
        fa.lane0 = ar_.at<int32_t>(o_final_lane0_);
        fa.nlanes = ar_.at<int32_t>(o_final_nl_);
        fa.obj = ar_.at<double>(o_final_obj_);
        fa.best_lane = ar_.at<int32_t>(o_final_best_);
        fa.x_out = ar_.at<uint8_t*>(o_final_xptr_);
        UBQP_CK(launch_finalize(fa, (int)ni, stream_));
        launches_ += 1;
        for (size_t t = 0; t < ni; ++t)
            if (xhost[t])
                UBQP_CK(cudaMemcpyAsync(x_out[t], xd[t], (size_t)inst_[t].n, cudaMemcpyDeviceToHost, stream_));
        if (is_device_ptr(obj_out))
            UBQP_CK(cudaMemcpyAsync(obj_out, fa.obj, ni * 8, cudaMemcpyDeviceToDevice, stream_));
        else
            UBQP_CK(cudaMemcpyAsync(obj_out, fa.obj, ni * 8, cudaMemcpyDeviceToHost, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        return UBQP_OK;
    }

    int states(std::vector<LaneState>& out)
    {
        out.resize(nlanes_);
        UBQP_CK(cudaMemcpyAsync(out.data(), ar_.at<LaneState>(o_states_), nlanes_ * sizeof(LaneState),
                                cudaMemcpyDeviceToHost, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        return UBQP_OK;
    }

    int fill_stats(ubqp_stats* s)
    {
        if (!s) return UBQP_OK;
        std::vector<LaneState> st;
        int rc = states(st);
        if (rc) return rc;
        memset(s, 0, sizeof(*s));
        for (int l = 0; l < nlanes_; ++l) {
            const LaneState& S = st[l];
            s->inner_iters += S.inner_iters;
            s->inner_steps += S.inner_steps;
            s->var_updates += S.inner_iters * (int64_t)lanes_[l].n;
            s->outer_steps += S.s;
            s->lobpcg_iters += S.lob_iters;
            s->jacobi_iters += S.jac_iters;
            s->floor_steps += S.floor_steps;
            s->lanes_capped += S.status == 1 ? 1 : 0;
            // the sparse minimum of the step's matrix-vector product (the stored entries of
            // Q_off as 4-byte values with 2-byte column indices, and 8 vectors of n floats)
            const int64_t nnz = (int64_t)nnz_host_[(size_t)lane_inst_[l]];
            s->alg_bytes += S.updates * (6 * nnz + 32 * (int64_t)lanes_[l].n);
            s->alg_flops += S.updates * 2 * nnz;
        }
        s->lanes = nlanes_;
        int64_t most = 0;
        for (const LaneState& S : st) most = std::max<int64_t>(most, S.updates);
        s->ticks = ticks_ >= 0 ? ticks_ : most;
        s->ms_device = ms_device_;
        s->phase_a_ms = phase_a_ms_;
        s->phase_a_launches = phase_a_launches_;
        unsigned long long by = 0;
        UBQP_CK(cudaMemcpyAsync(&by, ar_.at<unsigned long long>(o_bytes_), sizeof(by), cudaMemcpyDeviceToHost, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        s->phase_a_bytes = (int64_t)by;
        s->kernel_launches = launches_;
        s->ms_to_target = ms_to_target_;
        unsigned long long fl = 0;
        UBQP_CK(cudaMemcpyAsync(&fl, ar_.at<unsigned long long>(o_flops_), sizeof(fl), cudaMemcpyDeviceToHost, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        s->phase_a_flops = (int64_t)fl;
        s->cluster_size = tc_ ? tc_S_ : 0;
        s->cluster_tuned = cluster_tuned_;
        for (int c = 0; c < 9; ++c) s->cluster_probe_us[c] = cluster_probe_us_[c];
        s->tc_kernel = tc_ ? (tcp_ ? 2 : 1) : 0;
        s->sym_storage = sym_ ? 1 : 0;
        s->storage = tc_ ? 3 : (sparse_ ? 2 : (sym_ ? 1 : 0));
        s->gemv_kernel = tc_ ? 0 : (solo_ ? 3 : (loop_ ? 2 : 1));
        UBQP_CK(cudaMemcpyAsync(s->inner_hist, ar_.at<int64_t>(o_hist_), sizeof(s->inner_hist), cudaMemcpyDeviceToHost,
                                stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        return UBQP_OK;
    }

    int lane_vec_f64(int lane, int v, double* out_dev_or_host)
    {
        const int n = lanes_[lane].n;
        bool host = !is_device_ptr(out_dev_or_host);
        double* dst = out_dev_or_host;
        double* tmp = nullptr;
        AsyncTemp guard;
        if (host) {
            UBQP_CK(cudaMallocAsync((void**)&tmp, (size_t)n * 8, stream_));
            guard.hold(tmp, stream_);
            dst = tmp;
        }
        UBQP_CK(launch_lane_vec_to_f64(ar_.at<LaneDev>(o_lanes_), lane, v, n, dst, stream_));
        if (host) {
            UBQP_CK(cudaMemcpyAsync(out_dev_or_host, tmp, (size_t)n * 8, cudaMemcpyDeviceToHost, stream_));
            guard.release();
            UBQP_CK(cudaFreeAsync(tmp, stream_));
        }
        UBQP_CK(cudaStreamSynchronize(stream_));
        return UBQP_OK;
    }

    int trace_f64(int lane, int count_rows, double* tx, double* ta)
    {
        const int n = lanes_[lane].n;
        auto copy = [&](const float* src, double* dst, int64_t cnt) -> int {
            if (!dst || cnt <= 0) return UBQP_OK;
            bool host = !is_device_ptr(dst);
            double* d = dst;
            double* tmp = nullptr;
            AsyncTemp guard;
            if (host) {
                UBQP_CK(cudaMallocAsync((void**)&tmp, (size_t)cnt * 8, stream_));
                guard.hold(tmp, stream_);
                d = tmp;
            }
            UBQP_CK(launch_trace_to_f64(src, d, cnt, stream_));
            if (host) {
                UBQP_CK(cudaMemcpyAsync(dst, tmp, (size_t)cnt * 8, cudaMemcpyDeviceToHost, stream_));
                guard.release();
                UBQP_CK(cudaFreeAsync(tmp, stream_));
            }
            UBQP_CK(cudaStreamSynchronize(stream_));
            return UBQP_OK;
        };
        int rc = copy(ar_.at<float>(o_trace_x_[lane]), tx, (int64_t)count_rows * n);
        if (rc) return rc;
        return copy(ar_.at<float>(o_trace_a_[lane]), ta, count_rows);
    }

    int gamma_f64(int inst, double* out)
    {
        const size_t n = (size_t)inst_[inst].n;
        cudaMemcpyKind k = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        UBQP_CK(cudaMemcpyAsync(out, ar_.at<double>(inst_[inst].o_gamma), n * 8, k, stream_));
        UBQP_CK(cudaStreamSynchronize(stream_));
        return UBQP_OK;
    }

    bool inexact() const { return inexact_; }
    int64_t ticks() const { return ticks_; }
    double ms_device() const { return ms_device_; }
    int probe_ticks_ = 0;   // > 0: stop after about this many steps (restart tuner probes)

  private:
    ubqp_opts o_;
    bool tc_ = false;
    cudaStream_t stream_ = nullptr;
    cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t gexec_ = nullptr;
    int32_t* h_active_ = nullptr;
    int num_sms_ = 148;
    int max_ld_ = 32;
    int rows_per_item_ = 32;
    bool loop_ = false;          // FP32 lanes on the persistent lane loop
    bool solo_ = false;          // one FP32 lane on the single-lane persistent kernel
    bool sparse_ = false;        // FP32 lanes read Q'_off from the sliced row storage
    Arena sp_ar_;                // the sliced storage (allocated once its size is known)
    int64_t sliced_entries_ = 0;
    int solo_grid_ = 0, solo_nblk_ = 0;
    size_t o_solo_ = 0, o_sologrp_ = 0;
    std::vector<int32_t> solo_glanes_, solo_gfirst_, solo_gcta_, solo_tab_host_;
    std::vector<int> solo_nb_;   // row blocks per lane
    bool solo_one_ok_ = false;
    int solo_max_lanes_ = 1;
    int64_t solo_capc_ = 0;      // CTAs resident at once
    size_t solo_gmax_ = 1;       // groups the tables and barriers have room for
    int solo_nl_ = 0;            // lanes (the tables' first part)
    int loop_grid_ = 0, loop_budget_ = 0;
    uint64_t loop_cap_ = 0;
    int nitems_ = 0;
    int nlanes_ = 0;
    bool inexact_ = false;
    int64_t ticks_ = 0;
    double ms_device_ = 0.0;
    double phase_a_ms_ = 0.0;
    double ms_to_target_ = -1.0;
    unsigned long long tl_prev_ = 0;
    int64_t launches_ = 0;
    int64_t phase_a_launches_ = 0;
    std::vector<cudaEvent_t> evA_;
    Arena ar_;
    std::vector<InstDev> inst_;
    std::vector<LaneDev> lanes_;
    std::vector<LaneInit> lane_init_;
    std::vector<size_t> o_vec_, o_bx_, o_part_, o_trace_x_, o_trace_a_, o_x0_, o_p0_;
    size_t o_scal_ = 0, o_valid_ = 0, o_inexact_ = 0, o_hist_ = 0, o_active_ = 0, o_states_ = 0, o_lanes_ = 0,
           o_linit_ = 0, o_items_ = 0, o_bytes_ = 0, o_counters_ = 0, o_tcinst_ = 0, o_tcerr_ = 0, o_ring_ = 0, o_ht_ = 0, o_loopctr_ = 0, o_budget_ = 0,
           o_flops_ = 0, o_queue_ = 0;
    int tc_tiles_ = 0, tc_S_ = 1, tc_stages_ = 2, max_bn_ = 16;
    bool tcp_ = false;   // tensor-core lanes on the persistent kernel
    bool sym_ = false;   // FP32 lanes on the symmetric storage (lane loop only)
    std::vector<SymLane> sym_host_;
    std::vector<size_t> o_pbuf_;
    size_t o_symctr_ = 0, o_symlanes_ = 0;
    size_t ntact_total_ = 0, o_ntact_ = 0, o_row0_ = 0, o_valargs_ = 0, o_refargs_ = 0;
    std::vector<int32_t> ntact_host_;   // staged until the copy completes (the stream syncs in run)
    std::vector<unsigned long long> nnz_host_;   // stored off-diagonal entries per instance
    std::vector<int> lane_inst_;                 // instance of each lane
    size_t o_nnz_ = 0;
    int tcp_grid_ = 0;
    int cluster_tuned_ = 0;               // 0 rule or caller's choice, 1 measured now, 2 from the cache
    float cluster_probe_us_[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    size_t o_final_lane0_ = 0, o_final_nl_ = 0, o_final_obj_ = 0, o_final_best_ = 0, o_final_xptr_ = 0,
           o_final_xbuf_ = 0;
};

}  // namespace ubqp

// =====================================================================================
// C ABI
using namespace ubqp;

extern "C" {

void ubqp_opts_default(ubqp_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->method = UBQP_PABB;
    o->max_outer = 1000;
    o->max_inner = 10000;
    o->tol_inner = 1e-5;
    o->tol_outer = 1e-5;
    o->eta = 0.9;
    o->gamma_margin = 1.0;
    o->alpha_min = 1e-10;
    o->alpha_max = 1e10;
    o->tau_z = 1e-12;
    o->eps_hp_rel = 1e-8;
    o->lambda_floor_rel = 4.0;
    o->sigma_rel = 1e-3;
    o->seed = 0;
    o->restarts = 1;
    o->precision = UBQP_FP32;
    o->lobpcg_max_iter = 256;
    o->lobpcg_tol = 1e-7;
    o->jacobi_max_iter = 60;
    o->max_ticks_per_sync = 64;
    o->profile_kernels = 0;
    o->stop_at_target = 0;
    o->tc_cluster = 0;
    o->gemv_kernel = 0;
    o->lane_budget = 0;
    o->rows_per_item = 0;
    o->sym_storage = 1;
    o->wait_limit_us = 0;
    o->tc_fuse = 0;
    o->sparse_storage = 0;
    o->target_objective = INFINITY;
    o->stream = nullptr;
    o->mu = nullptr;
    o->x_starts = nullptr;
    o->stats = nullptr;
}

const char* ubqp_status_string(int s)
{
    switch (s) {
    case UBQP_OK: return "UBQP_OK";
    case UBQP_EINVAL: return "UBQP_EINVAL";
    case UBQP_ENOTSYM: return "UBQP_ENOTSYM";
    case UBQP_ENONFINITE: return "UBQP_ENONFINITE";
    case UBQP_ECUDA: return "UBQP_ECUDA";
    case UBQP_ENOMEM: return "UBQP_ENOMEM";
    case UBQP_ETIMEOUT: return "UBQP_ETIMEOUT";
    case UBQP_ENOTSUP: return "UBQP_ENOTSUP";
    case UBQP_EMAXITER: return "UBQP_EMAXITER";
    default: return "UBQP_UNKNOWN";
    }
}

const char* ubqp_last_error(void) { return g_last_error; }

int64_t ubqp_profile_timeline(float* ms_out, int64_t* work_out, int64_t cap)
{
    const int64_t n = (int64_t)g_tl_ms.size();
    const int64_t m = cap < n ? cap : n;
    for (int64_t i = 0; i < m; ++i) {
        if (ms_out) ms_out[i] = g_tl_ms[(size_t)i];
        if (work_out) work_out[i] = g_tl_work[(size_t)i];
    }
    return n;
}

// every instance's R lanes: start 0 from x^0 of Eq. (gamma) (Jacobi sweeps first), the
// others from the caller's starts or uniform draws in [0,1]^n
static std::vector<LaneIn> build_lanes(const std::vector<InstIn>& insts, int R)
{
    std::vector<LaneIn> lanes;
    lanes.reserve(insts.size() * (size_t)R);
    for (size_t t = 0; t < insts.size(); ++t)
        for (int r = 0; r < R; ++r) {
            LaneIn l;
            l.inst = (int)t;
            l.restart = r;
            l.phase = r == 0 ? PH_JACOBI : PH_EVAL;
            l.start_kind = r == 0 ? 0 : 1;
            l.x0 = (r > 0 && insts[t].starts) ? insts[t].starts + (size_t)(r - 1) * insts[t].n : nullptr;
            l.p0 = nullptr;
            l.stop_after = 0;
            l.trace_len = 0;
            lanes.push_back(l);
        }
    return lanes;
}

// Restart tuner: a 32-step probe of the real batch with each candidate count of starts per
// instance; the largest count whose step time is at most twice the single-start step time
// is returned.  Extra starts that leave the step time nearly unchanged (the step is bound by
// reading Q once, or by latency) improve the best objective at little cost; the tuner stops
// short of counts that would multiply the time of every step.
static int tune_restarts(const std::vector<InstIn>& insts, const ubqp_opts& o, bool tc, float* probe_us)
{
    static const int kCand[5] = {1, 8, 32, 64, 128};
    double t1 = 0.0;
    int best = 1;
    for (int c = 0; c < 5; ++c) {
        ubqp_opts po = o;
        po.restarts = kCand[c];
        po.stats = nullptr;
        po.profile_kernels = 0;
        po.stop_at_target = 0;
        po.target_objective = INFINITY;
        po.max_ticks_per_sync = 32;
        Solver S(po);
        S.probe_ticks_ = 32;
        std::vector<LaneIn> lanes = build_lanes(insts, kCand[c]);
        int rc = S.setup(insts, lanes, tc);
        if (rc == UBQP_ENOMEM) break;   // this many starts do not fit: keep the best so far
        if (rc) return rc;
        rc = S.run();
        if (rc) return rc;
        ubqp_stats st;
        rc = S.fill_stats(&st);
        if (rc) return rc;
        const double t = S.ms_device() / (double)std::max<int64_t>(st.ticks, 1);
        probe_us[c] = (float)(1e3 * t);
        if (c == 0) t1 = t;
        if (t <= 2.0 * t1) best = kCand[c];
    }
    return best;
}

int ubqp_solve_batched(int32_t num, const int64_t* n, const double* const* Q, const double* const* b,
                       const ubqp_opts* o_in, uint8_t* const* x_out, double* obj_out)
{
    auto t0 = std::chrono::steady_clock::now();
    g_last_error[0] = 0;
    if (num < 1 || !n || !Q || !x_out || !obj_out) {
        set_error("num >= 1 and non-null n, Q, x_out, obj_out are required");
        return UBQP_EINVAL;
    }
    ubqp_opts o;
    if (o_in) o = *o_in;
    else ubqp_opts_default(&o);
    for (int32_t t = 0; t < num; ++t) {
        if (n[t] < 1 || n[t] > 65536) { set_error("instance %d: n = %lld out of [1, 65536]", t, (long long)n[t]); return UBQP_EINVAL; }
        if (!Q[t] || !x_out[t]) { set_error("instance %d: null Q or x_out", t); return UBQP_EINVAL; }
    }
    const bool tc = o.precision != UBQP_FP32;
    std::vector<InstIn> insts(num);
    for (int32_t t = 0; t < num; ++t) {
        insts[t].n = n[t];
        insts[t].Q = Q[t];
        insts[t].b = b ? b[t] : nullptr;
        insts[t].mu = o.mu ? o.mu[t] : nullptr;
        insts[t].starts = o.x_starts ? o.x_starts[t] : nullptr;
        insts[t].reformulated = false;
    }
    int rc = check_opts(o);   // before the tuner, which builds lanes from these options
    if (rc) return rc;
    float probe_us[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (o.restarts == 0) {
        rc = tune_restarts(insts, o, tc, probe_us);
        if (rc < 0) return rc;
        o.restarts = rc;
    }
    std::vector<LaneIn> lanes = build_lanes(insts, o.restarts);
    Solver S(o);
    rc = S.setup(insts, lanes, tc);
    if (rc) return rc;
    rc = S.run();
    if (rc) return rc;
    rc = S.finalize(x_out, obj_out);
    if (rc) return rc;
    ubqp_stats st;
    rc = S.fill_stats(&st);
    if (rc) return rc;
    st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    st.restarts = o.restarts;
    for (int c = 0; c < 5; ++c) st.restart_probe_us[c] = probe_us[c];
    if (o.stats) *o.stats = st;
    return st.lanes_capped > 0 ? UBQP_EMAXITER : UBQP_OK;
}

int ubqp_solve(const double* Q, const double* b, int64_t n, const ubqp_opts* o, uint8_t* x_out, double* obj_out)
{
    const double* Qs[1] = {Q};
    const double* bs[1] = {b};
    uint8_t* xs[1] = {x_out};
    int64_t ns[1] = {n};
    return ubqp_solve_batched(1, ns, Qs, bs, o, xs, obj_out);
}

int ubqp_inner_run(const double* Qp, const double* bp, const double* p, const double* x0, int64_t n,
                   const ubqp_opts* o_in, int32_t trace_len, double* trace_x, double* trace_alpha, double* x_out,
                   int32_t* steps_out, int32_t* exit_out)
{
    g_last_error[0] = 0;
    if (n < 1 || n > 65536 || !Qp || !bp || !p || !x0 || trace_len < 0) {
        set_error("ubqp_inner_run: bad arguments");
        return UBQP_EINVAL;
    }
    ubqp_opts o;
    if (o_in) o = *o_in;
    else ubqp_opts_default(&o);
    o.precision = UBQP_FP32;
    o.restarts = 1;
    std::vector<InstIn> insts(1);
    insts[0] = InstIn{n, Qp, bp, nullptr, nullptr, true};
    std::vector<LaneIn> lanes(1);
    lanes[0] = LaneIn{0, 0, PH_INNER, 0, x0, p, STOP_INNER, trace_len};
    Solver S(o);
    int rc = S.setup(insts, lanes, false);
    if (rc) return rc;
    rc = S.run();
    if (rc) return rc;
    std::vector<LaneState> st;
    rc = S.states(st);
    if (rc) return rc;
    int rows = std::min<int>(trace_len, st[0].k + 1);
    if (trace_len > 0) {
        rc = S.trace_f64(0, rows, trace_x, trace_alpha);
        if (rc) return rc;
    }
    if (x_out) {
        rc = S.lane_vec_f64(0, V_X, x_out);
        if (rc) return rc;
    }
    if (steps_out) *steps_out = st[0].k;
    if (exit_out) *exit_out = st[0].last_exit;
    return UBQP_OK;
}

int ubqp_penalty_probe(const double* Qp, const double* bp, const double* p, const double* x, int64_t n,
                       const ubqp_opts* o_in, double* lambda_out, double* alpha_out, int32_t* n_active_out,
                       int32_t* iters_out)
{
    g_last_error[0] = 0;
    if (n < 1 || n > 65536 || !Qp || !bp || !p || !x) {
        set_error("ubqp_penalty_probe: bad arguments");
        return UBQP_EINVAL;
    }
    ubqp_opts o;
    if (o_in) o = *o_in;
    else ubqp_opts_default(&o);
    o.restarts = 1;
    if (o.max_outer < 1) o.max_outer = 1;
    std::vector<InstIn> insts(1);
    insts[0] = InstIn{n, Qp, bp, nullptr, nullptr, true};
    std::vector<LaneIn> lanes(1);
    lanes[0] = LaneIn{0, 0, PH_EVAL, 0, x, p, STOP_LOB, 0};
    Solver S(o);
    int rc = S.setup(insts, lanes, o.precision != UBQP_FP32);
    if (rc) return rc;
    rc = S.run();
    if (rc) return rc;
    std::vector<LaneState> st;
    rc = S.states(st);
    if (rc) return rc;
    if (lambda_out) *lambda_out = st[0].lam;
    if (alpha_out) *alpha_out = st[0].pen_alpha;
    if (n_active_out) *n_active_out = st[0].n_active;
    if (iters_out) *iters_out = (int32_t)st[0].lob_iters;
    return UBQP_OK;
}

int ubqp_initial_point(const double* Q, const double* b, const double* mu, int64_t n, const ubqp_opts* o_in,
                       double* x0_out, double* gamma_out)
{
    g_last_error[0] = 0;
    if (n < 1 || n > 65536 || !Q || !x0_out) {
        set_error("ubqp_initial_point: bad arguments");
        return UBQP_EINVAL;
    }
    ubqp_opts o;
    if (o_in) o = *o_in;
    else ubqp_opts_default(&o);
    o.precision = UBQP_FP32;
    o.restarts = 1;
    std::vector<InstIn> insts(1);
    insts[0] = InstIn{n, Q, b, mu, nullptr, false};
    std::vector<LaneIn> lanes(1);
    lanes[0] = LaneIn{0, 0, PH_JACOBI, 0, nullptr, nullptr, STOP_JACOBI, 0};
    Solver S(o);
    int rc = S.setup(insts, lanes, false);
    if (rc) return rc;
    rc = S.run();
    if (rc) return rc;
    rc = S.lane_vec_f64(0, V_X, x0_out);
    if (rc) return rc;
    if (gamma_out) rc = S.gamma_f64(0, gamma_out);
    return rc;
}

// the rows per work item of a gradient launch: the smallest power of two from 8 that keeps
// the items of all points within about 8 per SM (at most 256, one epilogue thread per row)
static int grad_rows_per_item(int64_t n, int64_t batch, int sms)
{
    int rb = 8;
    while (rb < 256 && batch * n / rb > 8 * (int64_t)sms) rb *= 2;
    return rb;
}

static int check_grad_args(const char* who, const void* Q, const void* b, const void* p, const void* x, int64_t n,
                           int64_t batch, int dtype, const void* h_out, const void* g_out, bool need_dev)
{
    if (!Q || !x || n < 1 || n > 65536 || batch < 1 || (dtype != UBQP_DTYPE_F32 && dtype != UBQP_DTYPE_F64)) {
        set_error("%s: need Q, x, 1 <= n <= 65536, batch >= 1 and dtype UBQP_DTYPE_F32 or UBQP_DTYPE_F64", who);
        return UBQP_EINVAL;
    }
    const uintptr_t es = dtype == UBQP_DTYPE_F64 ? 8 : 4;
    const void* ptrs[6] = {Q, b, p, x, h_out, g_out};
    for (const void* q : ptrs)
        if (q && (reinterpret_cast<uintptr_t>(q) % es) != 0) {
            set_error("%s: every pointer must be aligned to its element size", who);
            return UBQP_EINVAL;
        }
    if (need_dev)
        for (const void* q : ptrs)
            if (q && !is_device_ptr(q)) {
                set_error("%s: all pointers must be device memory", who);
                return UBQP_EINVAL;
            }
    return UBQP_OK;
}

int ubqp_penalized_eval(const void* Q, const void* b, const void* p, const void* x, int64_t n, int64_t batch,
                        int dtype, void* h_out, void* g_out, void* stream)
{
    g_last_error[0] = 0;
    int rc = check_grad_args("ubqp_penalized_eval", Q, b, p, x, n, batch, dtype, h_out, g_out, true);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = dtype == UBQP_DTYPE_F64 ? 8 : 4;
    if ((size_t)n * es > 227 * 1024) {
        set_error("ubqp_penalized_eval: one point (n = %lld) does not fit in shared memory", (long long)n);
        return UBQP_ENOTSUP;
    }
    int dev = 0, sms = 148;
    UBQP_CK(cudaGetDevice(&dev));
    UBQP_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int rb = grad_rows_per_item(n, batch, sms);
    const int64_t nblk = (n + rb - 1) / rb;
    if (batch * nblk > INT32_MAX) {
        set_error("ubqp_penalized_eval: batch x row blocks exceeds 2^31");
        return UBQP_EINVAL;
    }
    const size_t bytes_lanes = round_up((size_t)batch * sizeof(LaneDev), 256);
    const size_t bytes_items = round_up((size_t)(batch * nblk) * sizeof(int2), 256);
    const size_t bytes_queue = 256;
    const size_t bytes_part = (size_t)(batch * nblk) * sizeof(Partial);
    char* scratch = nullptr;
    UBQP_CK(cudaMallocAsync((void**)&scratch, bytes_lanes + bytes_items + bytes_queue + bytes_part, s));
    AsyncTemp guard;
    guard.hold(scratch, s);
    LaneDev* d_lanes = reinterpret_cast<LaneDev*>(scratch);
    int2* d_items = reinterpret_cast<int2*>(scratch + bytes_lanes);
    int32_t* d_queue = reinterpret_cast<int32_t*>(scratch + bytes_lanes + bytes_items);
    Partial* d_part = reinterpret_cast<Partial*>(scratch + bytes_lanes + bytes_items + bytes_queue);
    UBQP_CK(launch_grad_setup(d_lanes, d_items, d_queue, d_part, Q, b, p, x, g_out, (int)n, (int)batch, (int)nblk,
                              (int)es, s));
    TickArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.lanes = d_lanes;
    ta.items = d_items;
    ta.nitems = (int)(batch * nblk);
    ta.rows_per_item = rb;
    ta.nlanes = (int)batch;
    ta.max_ld = (int)n;
    ta.work = d_queue;
    ta.done = d_queue + 1;
    UBQP_CK(launch_phase_a_grad(ta, dtype, n, s));
    if (h_out) UBQP_CK(launch_grad_reduce(d_lanes, (int)batch, h_out, dtype, s));
    guard.release();
    UBQP_CK(cudaFreeAsync(scratch, s));
    UBQP_CK(cudaStreamSynchronize(s));
    return UBQP_OK;
}

int ubqp_penalized_vjp(const void* x, const void* g, const void* grad_h, int64_t n, int64_t batch, int dtype,
                       void* gx_out, void* gp_out, void* gb_out, void* stream)
{
    g_last_error[0] = 0;
    if (!x || !grad_h || (gx_out && !g) || n < 1 || batch < 1 || (dtype != UBQP_DTYPE_F32 && dtype != UBQP_DTYPE_F64)) {
        set_error("ubqp_penalized_vjp: need x, grad_h (and g when gx_out is set), n >= 1, batch >= 1 and a valid dtype");
        return UBQP_EINVAL;
    }
    const void* ptrs[6] = {x, g, grad_h, gx_out, gp_out, gb_out};
    for (const void* q : ptrs)
        if (q && !is_device_ptr(q)) {
            set_error("ubqp_penalized_vjp: all pointers must be device memory");
            return UBQP_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)stream;
    UBQP_CK(launch_penalized_vjp(x, g, grad_h, n, batch, dtype, gx_out, gp_out, gb_out, s));
    UBQP_CK(cudaStreamSynchronize(s));
    return UBQP_OK;
}

}  // extern "C"
