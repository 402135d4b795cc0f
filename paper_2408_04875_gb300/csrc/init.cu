// Set-up and tear-down kernels of the solver:
//   validate     symmetry / finiteness checks and max |Q| of the original data
//   reformulate  Sec. 3.5: symmetric perturbation mu (given, or drawn here), then
//                gamma_i = 2 sum_j |(Q+mu)_ij| + |b_i| + margin, Q' = Q + mu + Diag(gamma),
//                b' = b - gamma; stores Q'_off (FP32 or BF16), diag(Q'), row sums and the
//                original Q for the exact evaluation
//   lane_init    every lane's vectors and scalar state
//   finalize     per instance, the best lane (lowest objective, then lowest index) and
//                its rounded point
// Draws (perturbation, extra starts) use SplitMix64 (Steele, Lea & Flood 2014) keyed by
// (seed, instance, indices) and the Box-Muller transform for normal variates.
#include "ubqp_engine.cuh"

namespace ubqp {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t key4(uint64_t seed, uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ a);
    h = splitmix64(h ^ b);
    return splitmix64(h ^ c);
}

// uniform in (0, 1] from the top 53 bits
__device__ __forceinline__ double unit_open0(uint64_t h) { return ((double)(h >> 11) + 1.0) * 0x1.0p-53; }

__device__ __forceinline__ double normal_draw(uint64_t seed, uint64_t inst, uint64_t i, uint64_t j)
{
    double u1 = unit_open0(key4(seed, inst, i, j));
    double u2 = unit_open0(key4(seed ^ 0x5851F42D4C957F2Dull, inst, i, j));
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// ---------------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ float block_max(float v, float* sh)
{
    v = max_shfl_reduce(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x == 0) {
        for (int w = 0; w < NT / 32; ++w) r = fmaxf(r, sh[w]);
        sh[0] = r;
    }
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* sh)
{
    v = dsum_shfl_reduce(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < NT / 32; ++w) r += sh[w];
        sh[0] = r;
    }
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v)
{
    atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));  // v >= 0: int order = float order
}

// out[0] = max |Q_ij - Q_ji|, out[1] = max |Q_ij| (i != j), out[2] = nonfinite flag, out[3] = max|Q|
// and *nnz += the row's stored (nonzero) off-diagonal entries
__device__ __forceinline__ void validate_row(const double* __restrict__ Q, const double* __restrict__ b, int n,
                                             float* out, unsigned long long* nnz, int i)
{
    __shared__ float sh[8];
    float asym = 0.f, offmax = 0.f, qmax = 0.f, bad = 0.f;
    unsigned cnt = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double q = Q[(size_t)i * n + j];
        double qt = Q[(size_t)j * n + i];
        cnt += (j != i && q != 0.0) ? 1u : 0u;
        if (!isfinite(q)) bad = 1.f;
        float aq = (float)fabs(q);
        qmax = fmaxf(qmax, aq);
        if (j != i) offmax = fmaxf(offmax, aq);
        double dq = fabs(q - qt);
        asym = fmaxf(asym, isfinite(dq) ? (float)dq : 0.f);
    }
    if (threadIdx.x == 0 && b && !isfinite(b[i])) bad = 1.f;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nnz, (unsigned long long)cnt);
    asym = block_max<256>(asym, sh);
    offmax = block_max<256>(offmax, sh);
    bad = block_max<256>(bad, sh);
    qmax = block_max<256>(qmax, sh);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(out + 0, asym);
        atomic_max_nonneg(out + 1, offmax);
        atomic_max_nonneg(out + 2, bad);
        atomic_max_nonneg(out + 3, qmax);
    }
}

// one CTA per row i
__device__ __forceinline__ void reformulate_row(const RefArgs& a, int i)
{
    __shared__ double shd[8];
    __shared__ float shf[8];
    const int n = a.n, ld = a.ld;
    const double* Qrow = a.Q + (size_t)i * n;
    const double bi = a.b ? a.b[i] : 0.0;
    // perturbed row and its absolute sum
    double r = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double q = Qrow[j];
        double m = 0.0;
        bool touch = (j == i) || (!a.diag_only_mu);
        if (touch) {
            if (a.mu) m = a.mu[(size_t)i * n + j];
            else if (a.sigma > 0.0 && (q != 0.0 || j == i))
                m = a.sigma * normal_draw(a.seed, (uint64_t)a.inst, (uint64_t)min(i, j), (uint64_t)max(i, j));
        }
        double qm = q + m;
        r += fabs(qm);
    }
    r = block_sum_d<256>(r, shd);
    const double gam = a.no_gamma ? 0.0 : 2.0 * r + fabs(bi) + a.margin;  // Eq. (gamma), strict ">"
    // second pass: store Q'_off in the working precision and the off-diagonal row sum
    double oabs = 0.0, dii = 0.0;
    float offmax = 0.f;
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        double q = j < n ? Qrow[j] : 0.0;
        double m = 0.0;
        bool touch = (j == i) || (!a.diag_only_mu);
        if (j < n && touch) {
            if (a.mu) m = a.mu[(size_t)i * n + j];
            else if (a.sigma > 0.0 && (q != 0.0 || j == i))
                m = a.sigma * normal_draw(a.seed, (uint64_t)a.inst, (uint64_t)min(i, j), (uint64_t)max(i, j));
        }
        double qm = q + m;
        if (j == i) {
            dii = qm + gam;
            if (a.Qoff) a.Qoff[(size_t)i * ld + j] = 0.f;
            if (a.Qbf) a.Qbf[qbf_index(i, j, ld)] = __float2bfloat16_rn(0.f);
        } else {
            double stored;
            if (a.Qbf) {
                __nv_bfloat16 h = __float2bfloat16_rn((float)qm);
                a.Qbf[qbf_index(i, j, ld)] = h;
                stored = (double)__bfloat162float(h);
                if (j < n && stored != qm) atomicOr(a.inexact, 1);
            } else {
                float f = (float)qm;
                a.Qoff[(size_t)i * ld + j] = f;
                stored = (double)f;
            }
            oabs += fabs(stored);
            offmax = fmaxf(offmax, (float)fabs(stored));
        }
        if (a.Qeval) {
            float hi = (float)q;
            a.Qeval[(size_t)i * ld + j] = make_float2(hi, (float)(q - (double)hi));
        }
    }
    oabs = block_sum_d<256>(oabs, shd);
    offmax = block_max<256>(offmax, shf);
    // dii was set by exactly one thread; share it
    __shared__ double sh_dii;
    if (threadIdx.x == (i % blockDim.x)) sh_dii = dii;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double d = sh_dii;
        a.d[i] = (float)d;
        a.bprime[i] = (float)(bi - gam);
        a.tsum[i] = (float)(d - gam + bi);  // = (Q+mu)_ii + b_i: the gamma terms cancel exactly
        a.oabs[i] = (float)oabs;
        a.rabs[i] = (float)(oabs + fabs(d));
        if (a.gamma) a.gamma[i] = gam;
        if (a.borig) a.borig[i] = bi;
        if (a.qdb) a.qdb[i] = Qrow[i] + bi;
        atomic_max_nonneg(a.scal + 0, offmax);
        atomic_max_nonneg(a.scal + 1, (float)(oabs + fabs(d)));
    }
}

// the instance owning global row g of a batch: row0[t] <= g < row0[t + 1]
__device__ __forceinline__ int batch_instance(const int64_t* row0, int ninst, int64_t g)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row0[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// every instance of a batch in one launch: one CTA per row of every instance
__global__ void validate_kernel(const ValArgs* v, const int64_t* row0, int ninst)
{
    const int t = batch_instance(row0, ninst, blockIdx.x);
    const ValArgs& a = v[t];
    validate_row(a.Q, a.b, a.n, a.out, a.nnz, (int)(blockIdx.x - row0[t]));
}

__global__ void reformulate_kernel(const RefArgs* args, const int64_t* row0, int ninst)
{
    const int t = batch_instance(row0, ninst, blockIdx.x);
    reformulate_row(args[t], (int)(blockIdx.x - row0[t]));
}

// padding rows of the per-instance vectors (i in [n, ld)) are zero; one CTA per instance
__global__ void zero_tail_kernel(const RefArgs* args)
{
    const RefArgs& a = args[blockIdx.x];
    for (int i = a.n + threadIdx.x; i < a.ld; i += blockDim.x) {
        a.d[i] = 1.f;  // keeps divisions finite; never used for i >= n
        a.bprime[i] = 0.f;
        a.tsum[i] = 0.f;
        a.oabs[i] = 0.f;
        a.rabs[i] = 0.f;
        if (a.borig) a.borig[i] = 0.0;
        if (a.qdb) a.qdb[i] = 0.0;
    }
}

// one CTA per lane
__global__ void lane_init_kernel(LaneInitArgs a)
{
    const LaneDev& L = a.lanes[blockIdx.x];
    const LaneInit& I = a.init[blockIdx.x];
    const int n = L.n, ld = L.ld;
    float* vec = L.vec;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
        for (int v = 0; v < NVEC; ++v) vec[(size_t)v * ld + i] = 0.f;
        L.best_x[i] = 0;
        if (i >= n) {
            if (L.mode == MODE_TC) {
                L.u_hi[i] = __float2bfloat16_rn(0.f);
                if (L.u_lo) L.u_lo[i] = __float2bfloat16_rn(0.f);
            }
            continue;
        }
        float x;
        if (I.x0) x = (float)I.x0[i];
        else if (I.start_kind == 1)  // drawn start, uniform in [0, 1)
            x = (float)(unit_open0(key4(a.seed ^ 0xA0761D6478BD642Full, (uint64_t)I.inst, (uint64_t)I.restart,
                                        (uint64_t)i)) - 0x1.0p-53);
        else x = 0.5f;               // first Jacobi iterate for Eq. (gamma)
        float p = I.p0 ? (float)I.p0[i] : 0.f;
        vec[V_X * ld + i] = x;
        vec[V_P * ld + i] = p;
        vec[V_DMP * ld + i] = L.d[i] - p;
        vec[V_BBAR * ld + i] = L.bprime[i] + p;
        float u = (I.phase == PH_EVAL) ? (x > 0.5f ? 1.f : 0.f) : x;
        if (L.mode == MODE_TC) {
            __nv_bfloat16 hi = __float2bfloat16_rn(u);
            L.u_hi[i] = hi;
            if (L.u_lo) L.u_lo[i] = __float2bfloat16_rn(u - __bfloat162float(hi));
        } else {
            vec[V_U * ld + i] = u;
        }
    }
    if (threadIdx.x == 0) {
        LaneState S;
        memset(&S, 0, sizeof(S));
        S.phase = I.phase;
        S.best_f = INFINITY;
        S.best_s = -1;
        S.rho = 1.f;
        S.alpha = 1.f;
        *L.st = S;
    }
}

// one CTA per instance: best lane and its point
__global__ void finalize_kernel(FinalArgs a)
{
    const int inst = blockIdx.x;
    const int l0 = a.lane0[inst], R = a.nlanes[inst];
    __shared__ int best;
    if (threadIdx.x == 0) {
        int bl = l0;
        double bf = a.lanes[l0].st->best_f;
        for (int l = l0 + 1; l < l0 + R; ++l) {
            double f = a.lanes[l].st->best_f;
            if (f < bf) { bf = f; bl = l; }
        }
        best = bl;
        a.obj[inst] = bf;
        a.best_lane[inst] = bl - l0;
    }
    __syncthreads();
    const LaneDev& L = a.lanes[best];
    uint8_t* out = a.x_out[inst];
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) out[i] = L.best_x[i];
}

// FP32 copies of lane vectors for the test entry points
__global__ void lane_vec_to_f64_kernel(const LaneDev* lanes, int lane, int v, double* out)
{
    const LaneDev& L = lanes[lane];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x)
        out[i] = (double)L.vec[(size_t)v * L.ld + i];
}

__global__ void trace_to_f64_kernel(const float* in, double* out, int64_t count)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (double)in[t];
}

// ---------------------------------------------------------------------------------
// Packs Q'_off (n x ld FP32 rows, zero diagonal) into the upper-triangle tiles of the
// symmetric storage: kSymT x kSymT tiles (I, J), I <= J, row-major inside a tile, in the
// order (0,0), (0,1), .., (0,nb-1), (1,1), ...  One CTA per tile; rows beyond n are zero.
__global__ void pack_sym_kernel(const float* __restrict__ Qoff, int n, int ld, float* __restrict__ Qsym, int nb)
{
    int I = 0, rem = (int)blockIdx.x, rowlen = nb;
    while (rem >= rowlen) {
        rem -= rowlen;
        ++I;
        --rowlen;
    }
    const int J = I + rem;
    float* dst = Qsym + (size_t)blockIdx.x * kSymT * kSymT;
    for (int e = threadIdx.x; e < kSymT * kSymT; e += blockDim.x) {
        const int row = I * kSymT + e / kSymT, col = J * kSymT + e % kSymT;
        dst[e] = row < n ? Qoff[(size_t)row * ld + col] : 0.f;
    }
}

// ---------------------------------------------------------------------------------
// Sliced row storage of Q'_off (32-row slices): slice s holds, for k < width_s, the k-th
// stored entry of each of its 32 rows at entry spo[s] + 32 k + r (value, column); rows with
// fewer entries are padded with (0, column 0).  Built from the dense FP32 rows the
// reformulation wrote, so the stored entries are exactly the nonzero ones of Q'_off.

// stored entries per row, maximum per slice (one warp per row, a CTA per slice)
__global__ void sell_width_kernel(const float* __restrict__ Qoff, int n, int ld, int32_t* width)
{
    const int slice = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int wmax[8];
    int mx = 0;
    for (int r = warp; r < 32; r += 8) {
        const int row = slice * 32 + r;
        if (row >= n) continue;
        int cnt = 0;
        for (int c0 = 0; c0 < ld; c0 += 32) cnt += __popc(__ballot_sync(0xffffffffu, Qoff[(size_t)row * ld + c0 + lane] != 0.f));
        mx = max(mx, cnt);
    }
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int w = 0; w < 8; ++w) m = max(m, wmax[w]);
        width[slice] = m;
    }
}

// entries of each row in column order, one warp per row
__global__ void sell_pack_kernel(const float* __restrict__ Qoff, int n, int ld, const int64_t* __restrict__ spo,
                                 float* __restrict__ vals, uint16_t* __restrict__ cols)
{
    const int slice = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = spo[slice];
    const int width = (int)((spo[slice + 1] - base) / 32);
    for (int r = warp; r < 32; r += 8) {
        const int row = slice * 32 + r;
        int pos = 0;
        if (row < n) {
            for (int c0 = 0; c0 < ld; c0 += 32) {
                const float v = Qoff[(size_t)row * ld + c0 + lane];
                const unsigned m = __ballot_sync(0xffffffffu, v != 0.f);
                if (v != 0.f) {
                    const int p = pos + __popc(m & ((1u << lane) - 1u));
                    vals[base + (int64_t)p * 32 + r] = v;
                    cols[base + (int64_t)p * 32 + r] = (uint16_t)(c0 + lane);
                }
                pos += __popc(m);
            }
        }
        for (int p = pos + lane; p < width; p += 32) {
            vals[base + (int64_t)p * 32 + r] = 0.f;
            cols[base + (int64_t)p * 32 + r] = 0;
        }
    }
}

cudaError_t launch_sell_width(const float* Qoff, int n, int ld, int32_t* width, cudaStream_t s)
{
    sell_width_kernel<<<(n + 31) / 32, 256, 0, s>>>(Qoff, n, ld, width);
    return cudaGetLastError();
}

cudaError_t launch_sell_pack(const float* Qoff, int n, int ld, const int64_t* spo, float* vals, uint16_t* cols,
                             cudaStream_t s)
{
    sell_pack_kernel<<<(n + 31) / 32, 256, 0, s>>>(Qoff, n, ld, spo, vals, cols);
    return cudaGetLastError();
}

// stored (nonzero) off-diagonal entries of a device n x n FP64 matrix, added to *out
__global__ void count_offdiag_kernel(const double* __restrict__ Q, int n, unsigned long long* out)
{
    const int i = blockIdx.x;
    unsigned c = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) c += (j != i && Q[(size_t)i * n + j] != 0.0) ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

cudaError_t launch_count_offdiag(const double* Q, int n, unsigned long long* out, cudaStream_t s)
{
    count_offdiag_kernel<<<n, 256, 0, s>>>(Q, n, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_sym(const float* Qoff, int n, int ld, float* Qsym, cudaStream_t s)
{
    const int nb = ld / kSymT;
    pack_sym_kernel<<<nb * (nb + 1) / 2, 256, 0, s>>>(Qoff, n, ld, Qsym, nb);
    return cudaGetLastError();
}

cudaError_t launch_validate(const ValArgs* v, const int64_t* row0, int ninst, int64_t rows, cudaStream_t s)
{
    validate_kernel<<<(unsigned)rows, 256, 0, s>>>(v, row0, ninst);
    return cudaGetLastError();
}

cudaError_t launch_reformulate(const RefArgs* args, const int64_t* row0, int ninst, int64_t rows, cudaStream_t s)
{
    reformulate_kernel<<<(unsigned)rows, 256, 0, s>>>(args, row0, ninst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    zero_tail_kernel<<<ninst, 256, 0, s>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_lane_init(const LaneInitArgs& a, int nlanes, cudaStream_t s)
{
    lane_init_kernel<<<nlanes, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalArgs& a, int ninst, cudaStream_t s)
{
    finalize_kernel<<<ninst, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lane_vec_to_f64(const LaneDev* lanes, int lane, int v, int n, double* out, cudaStream_t s)
{
    lane_vec_to_f64_kernel<<<(n + 255) / 256, 256, 0, s>>>(lanes, lane, v, out);
    return cudaGetLastError();
}

cudaError_t launch_trace_to_f64(const float* in, double* out, int64_t count, cudaStream_t s)
{
    int blocks = (int)((count + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    trace_to_f64_kernel<<<blocks, 256, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

}  // namespace ubqp
