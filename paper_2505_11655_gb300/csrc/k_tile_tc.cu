// Tensor-core (tcgen05) variant of the float32 tiled likelihood kernel
// (arXiv:2505.11655 Sec. II A, Eq. (def:lnL:Decomposed), time-marginalised).
//
// Same decomposition as k_tile.cu: samples sorted by sky cell, a tile of 128 samples
// shares one Q window per (chunk of time bins, detector), the mode sum is contracted
// on the Q grid, R[s, c] = sum_r C[s, r] Qr[r, iw0 + c], then interpolated per bin.
// Here the contraction runs on the 5th-generation tensor cores:
//   * operands in float16 hi/lo pairs with power-of-two scaling (C rows per sample and
//     detector, Q by one global exponent), so that A_hi B_hi + A_hi B_lo + A_lo B_hi
//     carries ~22 significant bits, on par with the float32 contraction;
//   * A (128 x Kp, K-major) is written into shared memory by the prologue; B (128
//     columns x Kp, K-major) is a contiguous block of the pre-split Q copy, staged by
//     one TMA bulk copy per part into a double buffer;
//   * one thread issues 3 (Kp/16) tcgen05.mma.kind::f16 (M=128, N=128, K=16) into one
//     of two TMEM accumulators (128 columns each) and commits to an mbarrier;
//   * the block drains the accumulator with tcgen05.ld (warp quarter = 32 rows),
//     rescales, stores R to shared memory and gathers the two interpolation nodes of
//     every bin, while the next step's MMAs run.
// All waits are bounded (1 s by the global timer); a timeout raises kErrTimeout, the
// block abandons its tiles, frees its tensor memory and returns.
#include <cfloat>
#include <cmath>
#include <cuda_fp16.h>

#include "ile_kernels.h"
#include "tc_ptx.cuh"

namespace rift {

constexpr int kTcS = 128;          // samples per tile (MMA M)
constexpr int kTcW = 128;          // window columns per step (MMA N)
constexpr int kTcConsumers = 512;  // 16 consumer warps: drain, gather, log-sum-exp
constexpr int kTcThreads = kTcConsumers + 64;   // plus an MMA-issue warp and a TMA-staging warp
constexpr int kTcIssuerWarp = kTcConsumers / 32;
constexpr int kTcStagerWarp = kTcIssuerWarp + 1;
constexpr int kTcQ = kTcConsumers / kTcS;  // threads per sample in the gather (bin quarters)
constexpr int kTcBPT = 16;         // bins per thread per chunk
constexpr int kTcMaxBins = kTcQ * kTcBPT;
// phases B and E give every (sample, detector) item its own consumer thread, whole warps
// per detector
static_assert(kTcS * kMaxDet <= kTcConsumers && kTcS % 32 == 0, "one item per consumer thread");
// R is kept transposed, Rt[column][sample]: the drain (lane = sample, fixed column) and
// the gather (lane = sample, per-sample column) both touch bank = sample, conflict-free.
constexpr int kTcPow = 16;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr float kLog2e = 1.4426950408889634f;

// 2^x by the hardware approximation (PTX ex2.approx.ftz.f32: relative error ~2^-22,
// 0 for arguments below the float range)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// A tile whose samples span more than this many Q samples at some detector is cut
// into contiguous sub-groups (compact along the sort order) that are windowed apart.
constexpr int kTcSpreadLimit = 64;

struct TcLayout {
    size_t b, r, r2, tt, bins, i0, f0, inv, qsc, gid, lse, bar, tptr, end;
    size_t sky, e5, par, pw, pe, fx;   // prologue scratch, aliased on the B buffers
    int kp;
};

__host__ __device__ inline size_t tc_al(size_t o, size_t a = 128) { return (o + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int K, int M, int n_t)
{
    TcLayout L;
    L.kp = (2 * M + 15) / 16 * 16;
    size_t o = 0;
    L.b = o;
    const size_t bbytes = (size_t)2 * 2 * kTcW * L.kp * 2;
    // prologue scratch, every table sample-minor ([row][kTcS]) so that the lanes of a
    // warp (consecutive samples) touch consecutive words
    size_t s = L.b;
    L.sky = s;   s = tc_al(s + (size_t)3 * kTcS * 8, 16);
    L.e5 = s;    s = tc_al(s + (size_t)5 * kTcS * 4, 16);
    L.par = s;   s = tc_al(s + (size_t)4 * kTcS * 4, 16);
    L.pw = s;    s = tc_al(s + (size_t)2 * kTcPow * kTcS * 4, 16);
    L.pe = s;    s = tc_al(s + (size_t)(kMaxL + 1) * kTcS * 8, 16);
    L.fx = s;    s = tc_al(s + (size_t)K * kTcS * 8, 16);
    o = tc_al(L.b + (bbytes > s - L.b ? bbytes : s - L.b));
    // R tile; during the prologue it holds Y [M][kTcS] and, behind it, the template
    // matrices T_k (staged by a bulk copy at the start of every tile)
    L.r = o;
    L.tt = tc_al(L.r + (size_t)M * kTcS * 8);
    const size_t rbytes = (size_t)kTcW * kTcS * 4, pbytes = L.tt - L.r + (size_t)K * 2 * L.kp * L.kp * 2;
    o = tc_al(o + (rbytes > pbytes ? rbytes : pbytes));
    L.r2 = o;   // second R tile: steps alternate between the two
    o = tc_al(o + rbytes, 16);
    L.bins = o; o = tc_al(o + (size_t)n_t * 8, 16);   // (integer offset, fraction) per bin
    L.i0 = o;   o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.f0 = o;   o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.inv = o;  o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.qsc = o;  o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.gid = o;  o = tc_al(o + (size_t)kTcS * 4, 16);
    L.lse = o;  o = tc_al(o + (size_t)(2 * kTcQ + 2) * kTcS * 4, 16);
    L.bar = o;  o = tc_al(o + 8 * 8, 16);
    L.tptr = o; o = tc_al(o + 16, 16);
    L.end = o;
    return L;
}

bool lnl_tc_fits(const Problem &P, int max_smem)
{
    if (P.Qtc == nullptr || P.tc_groups <= 0)
        return false;
    const TcLayout L = tc_layout(P.K, P.M, P.n_t);
    // plus the kernel's static shared memory (sub-group table, ~5 KB)
    return L.kp <= 64 && L.end + 8192 <= (size_t)max_smem;
}

// ---------------------------------------------------------------- Q copy for the tensor path

__global__ void qmax_kernel(const double2 *__restrict__ Q64, int64_t count, unsigned int *qmax_bits)
{
    float m = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        double2 q = Q64[e];
        m = fmaxf(m, fmaxf(fabsf((float)q.x), fabsf((float)q.y)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f)
        atomicMax(qmax_bits, __float_as_uint(m));   // non-negative floats order as integers
}

// Global power-of-two exponent e with max|Q| 2^e in [2^13, 2^14).
__device__ __forceinline__ int q_exponent(unsigned int qmax_bits)
{
    float m = __uint_as_float(qmax_bits);
    if (!(m > 0.f))
        return 0;
    int ex;
    frexpf(m, &ex);   // m = f 2^ex, f in [0.5, 1)
    return 14 - ex;
}

// Qtc[k][part][group][kc][row][e]: group = 8 time columns, kc = 8 components.
__global__ void prep_tc_kernel(const double2 *__restrict__ Q64, int K, int M, int n_q, int groups, int kp,
                               const unsigned int *qmax_bits, __half *__restrict__ Qtc)
{
    const float scale = ldexpf(1.f, q_exponent(*qmax_bits));
    const int64_t per_part = (int64_t)groups * kp * 8;
    const int64_t total = (int64_t)K * per_part;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / per_part);
        const int64_t w = e - (int64_t)k * per_part;
        const int g = (int)(w / (kp * 8));
        const int rem = (int)(w - (int64_t)g * kp * 8);
        const int kc = rem / 64, row = (rem / 8) % 8, el = rem % 8;
        const int c = 8 * g + row, r = 8 * kc + el;
        float v = 0.f;
        if (c < n_q && r < 2 * M) {
            double2 q = Q64[((int64_t)k * M + r / 2) * n_q + c];
            v = (float)((r & 1) ? q.y : q.x) * scale;
        }
        const __half hi = __float2half_rn(v);
        const __half lo = __float2half_rn(v - __half2float(hi));
        __half *base = Qtc + (int64_t)k * 2 * per_part + w;
        base[0] = hi;
        base[per_part] = lo;
    }
}

cudaError_t launch_prep_tc(const double2 *Q64, int K, int M, int n_q, int groups, unsigned int *qmax_bits,
                           __half *Qtc, cudaStream_t st)
{
    const int kp = (2 * M + 15) / 16 * 16;
    cudaError_t e = cudaMemsetAsync(qmax_bits, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess)
        return e;
    const int64_t cnt = (int64_t)K * M * n_q;
    qmax_kernel<<<(int)std::min<int64_t>((cnt + 255) / 256, 1024), 256, 0, st>>>(Q64, cnt, qmax_bits);
    const int64_t tot = (int64_t)K * groups * kp * 8;
    prep_tc_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(Q64, K, M, n_q, groups, kp,
                                                                                  qmax_bits, Qtc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- template matrices

// One block per detector k.  With z = (Re c_0, Im c_0, Re c_1, ...) the template term of
// detector k is c^H U c + Re(c^T V c) = z^T T z with (U = Ur + i Ui, V = Vr + i Vi)
//   T[2a][2b] = Ur + Vr,  T[2a+1][2b+1] = Ur - Vr,  T[2a][2b+1] = -Ui - Vi,  T[2a+1][2b] = Ui - Vi
// (entries ab).  Stored transposed (row n = column n of T) as the B operand of W = Z T,
// scaled by 2^e with max|T| 2^e in [2^13, 2^14), float16 hi/lo, in the canonical K-major
// layout of the other operands.
__device__ __forceinline__ double tt_entry(const double2 *U, const double2 *V, int M, int r, int c)
{
    const int a = r >> 1, b = c >> 1;
    const double2 u = U[(size_t)a * M + b], v = V[(size_t)a * M + b];
    if (!(r & 1))
        return (c & 1) ? -u.y - v.y : u.x + v.x;
    return (c & 1) ? u.x - v.x : u.y - v.y;
}

__global__ void prep_tt_kernel(const double2 *__restrict__ U64, const double2 *__restrict__ V64, int M, int kp,
                               __half *__restrict__ Ttc, int *__restrict__ tt_exp)
{
    __shared__ float red[32];
    __shared__ int e_s;
    const int k = blockIdx.x, R2 = 2 * M;
    const double2 *U = U64 + (size_t)k * M * M, *V = V64 + (size_t)k * M * M;
    float m = 0.f;
    for (int e = threadIdx.x; e < R2 * R2; e += blockDim.x)
        m = fmaxf(m, fabsf((float)tt_entry(U, V, M, e / R2, e % R2)));
#pragma unroll
    for (int o = 16; o; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            mx = fmaxf(mx, red[w]);
        int ex = 0;
        if (mx > 0.f)
            frexpf(mx, &ex);
        e_s = mx > 0.f ? 14 - ex : 0;
        tt_exp[k] = e_s;
    }
    __syncthreads();
    const float sc = ldexpf(1.f, e_s);
    const int kc = kp / 8;
    __half *hi = Ttc + (size_t)k * 2 * kp * kp, *lo = hi + (size_t)kp * kp;
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
        const int n = e / kp, c = e % kp;   // row n of the operand = column n of T, component c
        const float v = (n < R2 && c < R2) ? (float)tt_entry(U, V, M, c, n) * sc : 0.f;
        const __half h = __float2half_rn(v);
        const size_t off = ((size_t)((n >> 3) * kc + (c >> 3)) * 8 + (n & 7)) * 8 + (c & 7);
        hi[off] = h;
        lo[off] = __float2half_rn(v - __half2float(h));
    }
}

cudaError_t launch_prep_tt(const double2 *U64, const double2 *V64, int K, int M, __half *Ttc, int *tt_exp,
                           cudaStream_t st)
{
    prep_tt_kernel<<<K, 256, 0, st>>>(U64, V64, M, (2 * M + 15) / 16 * 16, Ttc, tt_exp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- the kernel

// kDM: distance marginalisation (a separate instantiation, so that the plain path keeps
// its registers)
template <bool kDM>
__global__ void __launch_bounds__(kTcThreads, 1)
lnl_tc_kernel(Problem P, BinTable bt, const double *__restrict__ theta, const uint32_t *__restrict__ perm, int64_t n,
              double *__restrict__ lnL_tmarg, double *__restrict__ lnL_t, const double *__restrict__ lnpw,
              double *__restrict__ lnw, int *err, int *tile_counter, const uint32_t *__restrict__ n_dev,
              int64_t n_theta, int lnl_t_compact, PeakOut po)
{
    // n entries of perm (fewer when a device count is given, read where needed so that no
    // register holds it); every sample index in perm is below n_theta
    extern __shared__ __align__(128) unsigned char sm[];
    const int K = P.K, M = P.M, NT = P.n_t;
    const TcLayout L = tc_layout(K, M, NT);
    const int kp = L.kp, kcores = kp / 8;
    __half *Bs = reinterpret_cast<__half *>(sm + L.b);          // [2 buf][2 part][kTcW x kp]
    float *Rs = reinterpret_cast<float *>(sm + L.r);            // Rt [kTcW][kTcS] (prologue: Y [M][kTcS])
    float *Rs2 = reinterpret_cast<float *>(sm + L.r2);          // Rt of the odd steps
    int2 *bins = reinterpret_cast<int2 *>(sm + L.bins);          // (bin_i, bits of bin_f) per bin
    int *i0s = reinterpret_cast<int *>(sm + L.i0);              // [K][kTcS]
    float *f0s = reinterpret_cast<float *>(sm + L.f0);
    float *invs = reinterpret_cast<float *>(sm + L.inv);        // [K][kTcS] 2^-(row exponent + Q exponent)
    float *qsc = reinterpret_cast<float *>(sm + L.qsc);         // [K][kTcS] 2^-(2 row exponent)
    uint32_t *gid = reinterpret_cast<uint32_t *>(sm + L.gid);
    uint64_t *bbar = reinterpret_cast<uint64_t *>(sm + L.bar);  // [0,1] windows staged
    uint64_t *fullb = bbar + 2;   // [0,1] MMAs of an accumulator complete (tcgen05.commit)
    uint64_t *emptyb = bbar + 4;  // [0,1] accumulator drained by the 16 consumer warps
    uint64_t *tbar = bbar + 6;    // template matrices staged (once per tile)
    uint64_t *wbar = bbar + 7;    // template products W = Z T complete (once per tile)
    uint32_t *tptr = reinterpret_cast<uint32_t *>(sm + L.tptr);
    double *sky = reinterpret_cast<double *>(sm + L.sky);      // [3][kTcS] float64 unit vector n
    float *e5 = reinterpret_cast<float *>(sm + L.e5);          // [5][kTcS] sky basis of the response
    float *par = reinterpret_cast<float *>(sm + L.par);        // [cos 2psi, sin 2psi, D_ref/D][kTcS]
    float *pw = reinterpret_cast<float *>(sm + L.pw);          // [2 kTcPow][kTcS] cos^q, sin^q (iota/2)
    float2 *pe = reinterpret_cast<float2 *>(sm + L.pe);        // [kMaxL + 1][kTcS] exp(-i j phi)
    float2 *fx = reinterpret_cast<float2 *>(sm + L.fx);        // [K][kTcS] (D_ref/D) F_k
    float *lse = reinterpret_cast<float *>(sm + L.lse);         // [2][kTcQ][kTcS] running max, sum
    // [kTcS] per sample: the largest data term over its bins (order-preserving bits, high
    // word) and the first bin of the block of bins holding it (NT - bin, low word, so that
    // the lowest bin wins among equals), by one 64-bit shared atomic max per chunk and thread
    unsigned long long *peak = reinterpret_cast<unsigned long long *>(lse + 2 * kTcQ * kTcS);
    float *qsum = lse;                                          // [kTcQ][kTcS] template term partials
    float2 *Ys = reinterpret_cast<float2 *>(Rs);               // [M][kTcS] -2Y_lm(iota, -phi)
    __shared__ int lo_s[kMaxDet], hi_s[kMaxDet];        // current sub-group's offset range
    __shared__ int glo[kTcS][kMaxDet], ghi[kTcS][kMaxDet], gstart[kTcS + 1];
    __shared__ int tile_s, abort_s, ngroups_s;
    // bins per chunk for each sub-group offset spread (the float64 division once per block:
    // float64 is slow on this part)
    __shared__ int jmax_s[kTcSpreadLimit + 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double beta = P.t_step * P.fs;
    const int64_t n_tiles = ((n_dev ? min(n, (int64_t)*n_dev) : n) + kTcS - 1) / kTcS;
    const uint32_t idesc = tc::idesc_f16_f32(kTcS, kTcW);
    const uint32_t sbo = (uint32_t)kcores * 128u;
    const size_t part_halves = (size_t)kTcW * kp;                 // one B part
    const uint32_t part_bytes = (uint32_t)(part_halves * 2);
    const int qexp = q_exponent(*P.qmax_bits);
    // Shared-memory matrix descriptors (used by the issuer only; recomputed where used so
    // that nothing stays live in the other warps): the high word (stride byte offset,
    // version) is the same for every operand; the low word holds the start address and the
    // leading byte offset, so an operand offset is an addition to the address field (all
    // addresses < 256 KB: no carry out of it).
    auto desc = [&](uint32_t lo) { return ((uint64_t)(((sbo >> 4) & 0x3FFFu) | (1u << 14)) << 32) | lo; };
    auto desc_lo = [&](const void *p) { return ((tc::smem_u32(p) & 0x3FFFFu) >> 4) | ((128u >> 4) << 16); };
    // tensor memory columns: accumulators 0..255 (the template products W_k use columns
    // 64 k.. before the first window); the A operand (coefficients, float16 hi/lo, two
    // components per column) of detector k, part p at 256 + (2 k + p) kp / 2
    auto a_col = [&](int k, int part) { return 256u + (uint32_t)((2 * k + part) * (kp / 2)); };

    for (int j = tid; j < NT; j += blockDim.x) {
        bins[j] = make_int2(bt.bin_i[j], __float_as_int(bt.bin_f[j]));
    }
    // the nodes read for the bins j0 .. j0 + jmax - 1 lie within (jmax - 1) beta + 3 columns of
    // a sample's first node; with the spread of the sub-group's offsets and up to 7 columns of
    // window alignment that is at most kTcW - 1
    for (int sp = tid; sp <= kTcSpreadLimit; sp += blockDim.x) {
        const int jm = !(beta > 0.0) ? kTcMaxBins : (int)floor((double)(kTcW - 11 - sp) / beta) + 1;
        jmax_s[sp] = max(1, min(jm, kTcMaxBins));
    }
    if (warp == 0)
        tc::tmem_alloc(tptr, 512);
    if (tid == 0) {
        for (int i = 0; i < 4; ++i)
            tc::mbar_init(bbar + i, 1);
        for (int i = 4; i < 6; ++i)
            tc::mbar_init(bbar + i, kTcConsumers / 32);
        tc::mbar_init(tbar, 1);
        tc::mbar_init(wbar, 1);
        tc::fence_mbar_init();
        abort_s = 0;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tptr;
    // Barrier phase parities in one register (each role touches its own bits; bit b of a
    // field is buffer b): MMA completions awaited (consumers), windows consumed, accumulator
    // drains awaited and commits not yet matched by a drain wait (issuer), windows staged and
    // buffer staged at least once (stager), and the parity of the per-tile barriers (tbar,
    // wbar) over the tiles this block began.
    constexpr int kPhFull = 0, kPhCons = 2, kPhDrn = 4, kPhPend = 6, kPhStg = 8, kPhUsed = 10, kPhTile = 12;
    uint32_t ph = 0u;
    auto phbit = [&](int f, int b) { return (ph >> (f + b)) & 1u; };
    const bool producer = warp >= kTcIssuerWarp;   // issuer or stager

    for (;;) {
        // the R tile, written by this thread's drains, is the target of the next tile's bulk
        // copy of the template matrices
        tc::fence_proxy_async_smem();
        if (tid == 0)
            tile_s = abort_s ? INT_MAX : atomicAdd(tile_counter, 1);
        if (tid < kMaxDet) {
            lo_s[tid] = INT_MAX;
            hi_s[tid] = INT_MIN;
        }
        __syncthreads();
        const int64_t tile = tile_s;
        if (tile >= n_tiles)
            break;
        if (warp == kTcStagerWarp && lane == 0) {
            // template matrices into the tail of the R tile (free: the previous tile's last
            // gather is behind the barrier above)
            const uint32_t tt_bytes = (uint32_t)(K * 2 * kp * kp * 2);
            tc::mbar_expect_tx(tbar, tt_bytes);
            tc::bulk_g2s(sm + L.tt, P.Ttc, tt_bytes, tbar);
        }

        // ---------------- prologue A: sky trigonometry (float64) and per-sample scalars
        if (tid < kTcS) {
            const int64_t si = tile * kTcS + tid;
            const int64_t n_use = n_dev ? min(n, (int64_t)*n_dev) : n;
            uint32_t g = si < n_use ? perm[si] : 0xffffffffu;
            const bool valid = (int64_t)g < n_theta;
            gid[tid] = valid ? g : 0xffffffffu;
            peak[tid] = 0ull;
            double th[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
            if (valid)
                for (int d = 0; d < 6; ++d)
                    th[d] = theta[6 * (int64_t)g + d];
            Sky sk = sky_of(th[0], th[1], P.gmst);
            // unit vector to the source (Earth frame), float64 for the arrival delays
            sky[tid] = sk.cd * sk.ch;
            sky[kTcS + tid] = sk.cd * sk.sh;
            sky[2 * kTcS + tid] = sk.sd;
            // e_a = (-sin h, cos h, 0), e_d = (-sin d cos h, -sin d sin h, cos d), rounded once
            e5[tid] = (float)(-sk.sh);
            e5[kTcS + tid] = (float)sk.ch;
            e5[2 * kTcS + tid] = (float)(-sk.sd * sk.ch);
            e5[3 * kTcS + tid] = (float)(-sk.sd * sk.sh);
            e5[4 * kTcS + tid] = (float)sk.cd;
            float s2p, c2p, shalf, chalf, sphi, cphi;
            sincosf((float)(2.0 * th[2]), &s2p, &c2p);
            sincosf((float)(0.5 * th[4]), &shalf, &chalf);
            sincosf((float)th[3], &sphi, &cphi);
            par[tid] = c2p;
            par[kTcS + tid] = s2p;
            par[2 * kTcS + tid] = valid ? (kDM ? 1.f : (float)P.d_ref / (float)th[5]) : 0.f;
            float pc = 1.f, ps = 1.f;
            pw[tid] = 1.f;
            pw[kTcPow * kTcS + tid] = 1.f;
            for (int q = 1; q <= kMaxPow; ++q) {
                pc *= chalf;
                ps *= shalf;
                pw[q * kTcS + tid] = pc;
                pw[(kTcPow + q) * kTcS + tid] = ps;
            }
            // exp(-i j phi) for j = 0..kMaxL by repeated multiplication with exp(-i phi)
            float2 e = make_float2(1.f, 0.f);
            pe[tid] = e;
            for (int j = 1; j <= kMaxL; ++j) {
                e = make_float2(e.x * cphi + e.y * sphi, e.y * cphi - e.x * sphi);
                pe[j * kTcS + tid] = e;
            }
        }
        __syncthreads();
        // ---------------- B: delays, interpolation node split, x F_k
        for (int it = tid; tid < kTcConsumers && it < kTcS * K; it += kTcConsumers) {
            const int s = it % kTcS, k = it / kTcS;
            // Q-sample position of the first bin, (t_lo + dt_k - q_t0_k) fs
            const double u0 =
                fma(P.xfs[k][0], sky[s], fma(P.xfs[k][1], sky[kTcS + s], fma(P.xfs[k][2], sky[2 * kTcS + s], P.ufs0[k])));
            double fl = floor(u0);
            int i0 = (int)fl;
            i0s[k * kTcS + s] = i0;
            f0s[k * kTcS + s] = (float)(u0 - fl);
            // offset range of the tile at detector k: a warp holds 32 samples of one detector
            // (one item per thread), so reduce over the warp, then one atomic per warp
            const bool valid = gid[s] != 0xffffffffu;
            const int wmin = __reduce_min_sync(0xffffffffu, valid ? i0 : INT_MAX);
            const int wmax = __reduce_max_sync(0xffffffffu, valid ? i0 : INT_MIN);
            if (lane == 0 && wmin != INT_MAX) {
                atomicMin(&lo_s[k], wmin);
                atomicMax(&hi_s[k], wmax);
            }
            const Cx<float> F = response_f(P.Dten_f[k], e5[s], e5[kTcS + s], e5[2 * kTcS + s], e5[3 * kTcS + s],
                                           e5[4 * kTcS + s], par[s], par[kTcS + s]);
            const float amp = par[2 * kTcS + s];
            fx[k * kTcS + s] = make_float2(amp * F.re, amp * F.im);
        }
        // ---------------- C: harmonics Y_m = -2Y_lm(iota, -phi) [M][kTcS] (float32); the mode
        // coefficient of detector k is c_k,m = fx_k Y_m.  C reads only what A wrote, so it
        // follows B without a barrier (the float64 delays of B overlap the float32 work of C).
        for (int it = tid; tid < kTcConsumers && it < kTcS * M; it += kTcConsumers) {
            const int s = it % kTcS, m = it / kTcS;
            float d = 0.f;
            for (int t = 0; t < P.wn[m]; ++t)
                d += P.wcoef_f[m][t] * pw[P.wpc[m][t] * kTcS + s] * pw[(kTcPow + P.wps[m][t]) * kTcS + s];
            const int mm = P.mode_m[m];
            const float2 e = pe[(mm < 0 ? -mm : mm) * kTcS + s];   // exp(-i |m| phi)
            Ys[m * kTcS + s] = make_float2(d * e.x, d * (mm < 0 ? -e.y : e.y));
        }
        __syncthreads();
        // sub-groups: the whole tile when it is compact, else a greedy cut along the sort order
        if (tid == 0) {
            int spread = 0;
            for (int k = 0; k < K; ++k)
                spread = max(spread, hi_s[k] - lo_s[k]);
            int ng = 0;
            if (spread <= kTcSpreadLimit) {
                for (int k = 0; k < K; ++k) {
                    glo[0][k] = lo_s[k];
                    ghi[0][k] = hi_s[k];
                }
                gstart[0] = 0;
                ng = 1;
            } else {
                int lo[kMaxDet], hi[kMaxDet];
                bool open = false;
                for (int e = 0; e < kTcS; ++e) {
                    if (gid[e] == 0xffffffffu)
                        continue;   // padding rides along with the group it falls in
                    bool fits = open;
                    for (int k = 0; k < K && fits; ++k) {
                        const int v = i0s[k * kTcS + e];
                        fits = max(hi[k], v) - min(lo[k], v) <= kTcSpreadLimit;
                    }
                    if (!fits) {
                        if (open) {
                            for (int k = 0; k < K; ++k) {
                                glo[ng][k] = lo[k];
                                ghi[ng][k] = hi[k];
                            }
                            ++ng;
                        }
                        gstart[ng] = ng == 0 ? 0 : e;
                        for (int k = 0; k < K; ++k)
                            lo[k] = hi[k] = i0s[k * kTcS + e];
                        open = true;
                    } else {
                        for (int k = 0; k < K; ++k) {
                            lo[k] = min(lo[k], i0s[k * kTcS + e]);
                            hi[k] = max(hi[k], i0s[k * kTcS + e]);
                        }
                    }
                }
                for (int k = 0; k < K; ++k) {
                    glo[ng][k] = open ? lo[k] : 0;
                    ghi[ng][k] = open ? hi[k] : 0;
                }
                ++ng;
            }
            gstart[ng] = kTcS;
            ngroups_s = ng;
        }
        // ---------------- E: A operand, float16 hi/lo with a power-of-two scale per (sample,
        // detector), written into tensor memory: the thread of sample s writes lane s (its
        // warp's lane quarter), 16 components (8 columns) per store.  The previous tile's MMAs,
        // the last readers of these columns, completed before the barriers above.
        {
            tc::tc_fence_after();
            for (int it = tid; tid < kTcConsumers && it < kTcS * K; it += kTcConsumers) {
                const int s = it % kTcS, k = it / kTcS;
                const float2 f = fx[k * kTcS + s];
                float mx = 0.f;
                for (int m = 0; m < M; ++m) {
                    const float2 y = Ys[m * kTcS + s];
                    mx = fmaxf(mx, fmaxf(fabsf(f.x * y.x - f.y * y.y), fabsf(f.x * y.y + f.y * y.x)));
                }
                int ex = 0;
                if (mx > 0.f)
                    frexpf(mx, &ex);
                const int es = mx > 0.f ? 14 - ex : 0;
                const float sc = ldexpf(1.f, es);
                invs[k * kTcS + s] = ldexpf(1.f, -es - qexp);
                qsc[k * kTcS + s] = ldexpf(1.f, -es);
                const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
                for (int kk = 0; kk < kp / 16; ++kk) {
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int m = 8 * kk + j;
                        float cr = 0.f, ci = 0.f;
                        if (m < M) {
                            const float2 y = Ys[m * kTcS + s];
                            cr = (f.x * y.x - f.y * y.y) * sc;
                            ci = (f.x * y.y + f.y * y.x) * sc;
                        }
                        const __half hr = __float2half_rn(cr), hi = __float2half_rn(ci);
                        const __half lr = __float2half_rn(cr - __half2float(hr));
                        const __half li = __float2half_rn(ci - __half2float(hi));
                        hw[j] = (uint32_t)__half_as_ushort(hr) | ((uint32_t)__half_as_ushort(hi) << 16);
                        lw[j] = (uint32_t)__half_as_ushort(lr) | ((uint32_t)__half_as_ushort(li) << 16);
                    }
                    tc::tmem_st8(lane_base + a_col(k, 0) + 8u * (uint32_t)kk, hw);
                    tc::tmem_st8(lane_base + a_col(k, 1) + 8u * (uint32_t)kk, lw);
                }
                tc::tmem_st_wait();
            }
            tc::tc_fence_before();
        }
        // the prologue scratch (generic accesses above) shares its bytes with the B buffers,
        // which the stager refills by bulk copies (async proxy) once the steps begin
        tc::fence_proxy_async_smem();
        __syncthreads();

        // gather / fold ownership: thread -> sample s, bin quarter h of every chunk
        const int gs = tid & (kTcS - 1), gh = (tid >> 7) & (kTcQ - 1);
        const bool gok = !producer && gid[gs] != 0xffffffffu;

        // ---------------- D: template term on the tensor cores.  W_k = Z_k T_k (Z_k: the A
        // operand, row s = 2^es_ks z_ks rounded to float16 hi/lo; T_k scaled by 2^e_k), into the
        // accumulator columns 64 k.. (free until the first window's MMAs, which follow the
        // barrier below), then with the float32 components z_ks
        //   z_ks^T T_k z_ks = 2^-(es_ks + e_k) sum_n z_ks[n] W_k[s][n].
        int wfail = 0;
        if (warp == kTcIssuerWarp) {
            if (lane == 0) {
                if (!tc::mbar_wait(tbar, phbit(kPhTile, 0), kWaitNs)) {
                    wfail = 1;
                } else {
                    tc::tc_fence_after();
                    const uint32_t wdesc = tc::idesc_f16_f32(kTcS, kp);
                    const uint32_t t_lo0 = desc_lo(sm + L.tt);
                    const uint32_t t_part = (uint32_t)(kp * kp * 2) >> 4;
                    for (int k = 0; k < K; ++k) {
                        const uint32_t d = tmem + 64u * (uint32_t)k;
                        const uint32_t ah = tmem + a_col(k, 0), al = tmem + a_col(k, 1);
                        const uint32_t th = t_lo0 + (uint32_t)(2 * k) * t_part, tl = th + t_part;
                        for (int kk = 0; kk < kp / 16; ++kk) {
                            const uint32_t o = (uint32_t)kk * 16u, oa = (uint32_t)kk * 8u;
                            // all four hi/lo products (the template term is cheap on the tensor pipe)
                            tc::mma_f16_ta(d, ah + oa, desc(th + o), wdesc, kk > 0);
                            tc::mma_f16_ta(d, ah + oa, desc(tl + o), wdesc, 1);
                            tc::mma_f16_ta(d, al + oa, desc(th + o), wdesc, 1);
                            tc::mma_f16_ta(d, al + oa, desc(tl + o), wdesc, 1);
                        }
                    }
                    tc::mma_commit(wbar);
                }
            }
            wfail = __shfl_sync(0xffffffffu, wfail, 0);
        } else if (!producer) {
            // warp (q, cb) drains 16-column chunks cb, cb + 4, ... of the K W tiles for the
            // 32 samples of its lane quarter q
            const int ok = tc::mbar_wait(wbar, phbit(kPhTile, 0), kWaitNs) ? 1 : 0;
            tc::tc_fence_after();
            const int q = warp & 3, cb = warp >> 2, s = 32 * q + lane;
            float qp = 0.f;
            if (ok) {
                const int cpd = kp / 16;
                for (int c = cb; c < K * cpd; c += 4) {
                    const int k = c / cpd, n0 = (c - k * cpd) * 16;
                    uint32_t v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 64u * (uint32_t)k + (uint32_t)n0, v);
                    const float2 f = fx[k * kTcS + s];
                    tc::tmem_ld_wait();
                    float acc = 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {   // modes n0 / 2 + j: components (re, im)
                        const int m = n0 / 2 + j;
                        if (m < M) {
                            const float2 y = Ys[m * kTcS + s];
                            acc = fmaf(f.x * y.x - f.y * y.y, __uint_as_float(v[2 * j]), acc);
                            acc = fmaf(f.x * y.y + f.y * y.x, __uint_as_float(v[2 * j + 1]), acc);
                        }
                    }
                    qp += acc * ldexpf(qsc[k * kTcS + s], -P.tt_exp[k]);
                }
            }
            qsum[cb * kTcS + s] = qp;
            wfail = !ok;
        }
        tc::tc_fence_before();
        int failed = __syncthreads_or(wfail);
        ph ^= 1u << kPhTile;
        const float gqd =
            (float)P.kappa * ((qsum[gs] + qsum[kTcS + gs]) + (qsum[2 * kTcS + gs] + qsum[3 * kTcS + gs]));
        float run_mx = -INFINITY, run_sum = 0.f;
        const int ngroups = ngroups_s;
        for (int grp = 0; grp < ngroups && !failed; ++grp) {
            int spread = 0;
            for (int k = 0; k < K; ++k)
                spread = max(spread, ghi[grp][k] - glo[grp][k]);
            const bool in_grp = gs >= gstart[grp] && gs < gstart[grp + 1];
            // a sub-group's spread never exceeds kTcSpreadLimit (the cut above); the float64
            // expression is kept for the case that cannot occur
            int jmax = spread <= kTcSpreadLimit ? jmax_s[spread]
                                                : (!(beta > 0.0) ? kTcMaxBins : (int)floor((double)(kTcW - 11 - spread) / beta) + 1);
            jmax = max(1, min(jmax, kTcMaxBins));
            const int n_chunks = (NT + jmax - 1) / jmax;
            const int jnom = (NT + n_chunks - 1) / n_chunks;
            const int n_steps = n_chunks * K;
            // Step t covers detector t % K and the bins of chunk t / K (both tracked as
            // counters).  First Q column of the window of detector k for the chunk starting at
            // bin j0, clamped so that a window never leaves the allocation of the Q copy.
            auto win0 = [&](int k, int j0) {
                return min(max(glo[grp][k] + bins[j0].x, 0), 8 * (P.tc_groups - 16)) & ~7;
            };

            if (warp == kTcIssuerWarp) {
                // ============ issuer warp, lane 0: one MMA batch per staged window
                if (lane == 0) {
                    const uint32_t b_lo0 = desc_lo(Bs), b_part = part_bytes >> 4;
                    int k = 0;
                    for (int t = 0; t < n_steps && !failed; ++t, k = k + 1 == K ? 0 : k + 1) {
                        const int b = t & 1;
                        // window t staged; accumulator b drained by the consumers
                        if (!tc::mbar_wait(bbar + b, phbit(kPhCons, b), kWaitNs) ||
                            (phbit(kPhPend, b) && !tc::mbar_wait(emptyb + b, phbit(kPhDrn, b), kWaitNs))) {
                            failed = 1;
                            break;
                        }
                        ph ^= 1u << (kPhCons + b);
                        if (phbit(kPhPend, b))
                            ph ^= 1u << (kPhDrn + b);
                        tc::tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(b * kTcW);
                        const uint32_t ah = tmem + a_col(k, 0), al = tmem + a_col(k, 1);
                        const uint32_t bh = b_lo0 + (uint32_t)(2 * b) * b_part, bl = bh + b_part;
                        for (int kk = 0; kk < kp / 16; ++kk) {
                            const uint32_t o = (uint32_t)kk * 16u;   // 256 bytes: the next 16 components
                            const uint32_t oa = (uint32_t)kk * 8u;   // 16 components = 8 columns of A
                            tc::mma_f16_ta(d, ah + oa, desc(bh + o), idesc, kk > 0);
                            tc::mma_f16_ta(d, ah + oa, desc(bl + o), idesc, 1);
                            tc::mma_f16_ta(d, al + oa, desc(bh + o), idesc, 1);
                        }
                        tc::mma_commit(fullb + b);
                        ph |= 1u << (kPhPend + b);
                    }
                    if (failed)
                        abort_s = 1;
                }
                __syncwarp();
            } else if (warp == kTcStagerWarp) {
                // ============ stager warp, lane 0: windows into the two B buffers.  Every
                // window staged into buffer b is consumed by exactly one MMA batch that commits
                // to fullb[b], so before the j-th window into b the stager waits for the
                // (j - 1)-th completion of fullb[b] (that of the previous group or tile when
                // this is a group's first window into b).
                if (lane == 0) {
                    int sk = 0, sch = 0;   // detector and chunk of the next window
                    for (int t = 0; t < n_steps && !failed; ++t) {
                        const int b = t & 1;
                        if (phbit(kPhUsed, b) && !tc::mbar_wait(fullb + b, phbit(kPhStg, b) ^ 1u, kWaitNs)) {
                            failed = 1;
                            break;
                        }
                        const int g0 = win0(sk, sch * jnom) >> 3;
                        const __half *src = P.Qtc + ((size_t)sk * 2 * P.tc_groups + g0) * (size_t)kp * 8;
                        __half *dst = Bs + (size_t)b * 2 * part_halves;
                        tc::mbar_expect_tx(bbar + b, 2 * part_bytes);
                        tc::bulk_g2s(dst, src, part_bytes, bbar + b);
                        tc::bulk_g2s(dst + part_halves, src + (size_t)P.tc_groups * kp * 8, part_bytes, bbar + b);
                        ph ^= 1u << (kPhStg + b);
                        ph |= 1u << (kPhUsed + b);
                        if (++sk == K) {
                            sk = 0;
                            ++sch;
                        }
                    }
                    if (failed)
                        abort_s = 1;
                }
                __syncwarp();
            } else {
                // ============ consumer warps: drain, gather, fold
                float lin[kTcBPT], bfj[kTcBPT];
                int bj[kTcBPT];
#pragma unroll
                for (int i = 0; i < kTcBPT; ++i) {
                    lin[i] = 0.f;
                    bfj[i] = 0.f;
                    bj[i] = 0;
                }
                for (int t = 0, k = 0, j0 = 0; t < n_steps; ++t) {
                    const int b = t & 1, J = min(jnom, NT - j0);
                    const int jq = (J + kTcQ - 1) / kTcQ;                 // bins per quarter
                    const int jb = j0 + gh * jq, jn = max(0, min(jq, j0 + J - jb));   // this thread's bins
                    // every lane waits for the MMAs of step t (the same barrier word: no
                    // divergent branch, no broadcast of the result)
                    const int ok = tc::mbar_wait(fullb + b, phbit(kPhFull, b), kWaitNs) ? 1 : 0;
                    ph ^= 1u << (kPhFull + b);
                    tc::tc_fence_after();
                    // The rows of sample quarter q (TMEM lanes 32q..) are drained and gathered by
                    // the same four warps (warp & 3 == q), which synchronise on their own barrier
                    // once per step, after the drain.  Steps alternate between two R tiles: the
                    // tile step t drains into was last read by the gathers of step t - 2, which
                    // every warp of the quarter finished before the barrier of step t - 1.
                    const int qbar = 2 + (warp & 3);
                    float *Rt = (t & 1) ? Rs2 : Rs;
                    // The gather's own loads do not depend on the drain: issued before it, their
                    // shared-memory latency overlaps the drain.  Padding samples and samples of
                    // other sub-groups read at the group's lowest offset, which keeps every read
                    // in the row; their sums are discarded.
                    const int iw0 = win0(k, j0);
                    const bool mine = gok && in_grp;
                    const float *Rcol = Rt + ((mine ? i0s[k * kTcS + gs] : glo[grp][k]) - iw0) * kTcS + gs;
                    const float ff = mine ? f0s[k * kTcS + gs] : 0.f;
                    const float sc = invs[k * kTcS + gs];
                    if (k == 0) {
                        // this thread's bins of the chunk, shared by every detector (idle slots
                        // re-read the quarter's last bin, so that they repeat its value, or a
                        // valid bin when the quarter has none; one 8-byte broadcast load each)
                        const int jl = jn > 0 ? jb + jn - 1 : min(jb, NT - 1);
#pragma unroll
                        for (int i = 0; i < kTcBPT; ++i) {
                            const int j = min(jb + i, jl);
                            const int2 bv = bins[j];
                            bj[i] = bv.x;
                            bfj[i] = __int_as_float(bv.y);
                        }
                    }
                    {
                        // drain accumulator b: warp quarter q = rows 32q.., column block w / 4 of 32
                        const int q = warp & 3, cb = warp >> 2;
                        float *Rcol = Rt + (32 * cb) * kTcS + 32 * q + lane;
                        // two loads of 16 columns (fewer live registers than one of 32)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            uint32_t v[16];
                            tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTcW + 32 * cb + 16 * h), v);
                            tc::tmem_ld_wait();
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                Rcol[(16 * h + i) * kTcS] = __uint_as_float(v[i]);
                        }
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    tc::mbar_arrive_if(emptyb + b, lane == 0);
                    // this quarter's rows of R complete; agree on failure
                    if (tc::named_bar_or(qbar, kTcConsumers / 4, !ok || abort_s)) {
                        failed = 1;
                        break;
                    }
                    // two bins per packed float32 operation (the same roundings as one at a time)
#pragma unroll
                    for (int i = 0; i < kTcBPT; i += 2) {
                        const float2 sf = __fadd2_rn(make_float2(ff, ff), make_float2(bfj[i], bfj[i + 1]));
                        const int c0 = sf.x >= 1.f, c1 = sf.y >= 1.f;
                        const float2 fr = __fadd2_rn(sf, make_float2(-(float)c0, -(float)c1));
                        const float *ra = Rcol + (bj[i] + c0) * kTcS, *rb = Rcol + (bj[i + 1] + c1) * kTcS;
                        const float2 r0 = make_float2(ra[0], rb[0]), r1 = make_float2(ra[kTcS], rb[kTcS]);
                        const float2 v = __ffma2_rn(fr, __fadd2_rn(r1, make_float2(-r0.x, -r0.y)), r0);
                        const float2 l = __ffma2_rn(make_float2(sc, sc), v, make_float2(lin[i], lin[i + 1]));
                        lin[i] = l.x;
                        lin[i + 1] = l.y;
                    }
                    if (k == K - 1) {
                        // fold this thread's bins of the chunk into its running log-sum-exp
                        float cmx = -INFINITY;
                        if (kDM) {
                            // distance marginal per bin: a cheap upper bound first; the bin
                            // with the highest bound is evaluated, and a bin whose bound lies
                            // more than 40 below the larger of that value and the running
                            // maximum cannot move the marginal (< e^-40): left out
                            // (the bound is recomputed in the second loop rather than kept: it is
                            // a handful of operations, a register array of it is not)
                            float bmax = -INFINITY, abest = 0.f;
#pragma unroll
                            for (int i = 0; i < kTcBPT; ++i) {
                                const float bd = i < jn ? dm_bound32(P, lin[i], gqd) : -INFINITY;
                                if (bd > bmax) {
                                    bmax = bd;
                                    abest = lin[i];
                                }
                            }
                            const float vbest = jn > 0 ? ln_dist_marg32(P, abest, gqd) : -INFINITY;
                            // (every bin exact when the per-bin values are written out)
                            const float thr = lnL_t ? -INFINITY : fmaxf(run_mx, vbest) - 40.f;
#pragma unroll
                            for (int i = 0; i < kTcBPT; ++i) {
                                lin[i] = (i < jn && dm_bound32(P, lin[i], gqd) >= thr) ? ln_dist_marg32(P, lin[i], gqd)
                                                                                      : -INFINITY;
                                if (i < jn)
                                    cmx = fmaxf(cmx, lin[i]);
                            }
                        } else {
                            // lin holds the data term; ln L = lin - gqd, the template term
                            // subtracted once per sample in the epilogue (in float64)
                            // (the maximum by blocks of kPeakBlockTc bins, the same number of
                            // operations, so that the block holding it is known).  Idle slots
                            // repeat the last bin's value: the maximum is that of the valid
                            // bins, and the lowest block attaining it holds a valid bin.
                            float qm[kTcBPT / kPeakBlockTc];
#pragma unroll
                            for (int a = 0; a < kTcBPT / kPeakBlockTc; ++a) {
                                qm[a] = lin[kPeakBlockTc * a];
#pragma unroll
                                for (int i = kPeakBlockTc * a + 1; i < kPeakBlockTc * (a + 1); ++i)
                                    qm[a] = fmaxf(qm[a], lin[i]);
                            }
                            const float m01 = fmaxf(qm[0], qm[1]), m23 = fmaxf(qm[2], qm[3]);
                            cmx = fmaxf(m01, m23);
                            if (jn > 0 && in_grp) {
                                const int a = m01 >= m23 ? (qm[0] >= qm[1] ? 0 : 1) : (qm[2] >= qm[3] ? 2 : 3);
                                const uint32_t ob = __float_as_uint(cmx) ^
                                                    ((uint32_t)((int)__float_as_uint(cmx) >> 31) | 0x80000000u);
                                atomicMax(peak + gs,
                                          ((unsigned long long)ob << 32) | (unsigned)(NT - jb - kPeakBlockTc * a));
                            }
                        }
                        if (lnL_t && gok && in_grp) {
                            for (int i = 0; i < jn; ++i)
#pragma unroll
                                for (int u = 0; u < kTcBPT; ++u)
                                    if (u == i)
                                        lnL_t[(lnl_t_compact ? (int64_t)tile_s * kTcS + gs : (int64_t)gid[gs]) * NT + jb + i] =
                                            kDM ? (double)lin[u] : (double)lin[u] - (double)gqd;
                        }
                        if (jn > 0 && in_grp) {
                            const float nm = fmaxf(run_mx, cmx);
                            float cs = 0.f;
                            if (kDM) {
#pragma unroll
                                for (int i = 0; i < kTcBPT; ++i)
                                    if (i < jn)
                                        cs += __expf(lin[i] - nm);
                            } else {
                                // exp(lin - nm) = 2^(lin log2(e) - nm log2(e)), two bins per packed
                                // operation
                                const float off = nm * kLog2e;
                                float2 cs2 = make_float2(0.f, 0.f);
#pragma unroll
                                for (int i = 0; i < kTcBPT; i += 2) {
                                    const float2 x = __ffma2_rn(make_float2(lin[i], lin[i + 1]), make_float2(kLog2e, kLog2e),
                                                                make_float2(-off, -off));
                                    const float2 ev = make_float2(i < jn ? ex2_approx(x.x) : 0.f,
                                                                  i + 1 < jn ? ex2_approx(x.y) : 0.f);
                                    cs2 = __fadd2_rn(cs2, ev);
                                }
                                cs = cs2.x + cs2.y;
                            }
                            run_sum = (run_mx == -INFINITY ? 0.f : run_sum * __expf(run_mx - nm)) + cs;
                            run_mx = nm;
                        }
#pragma unroll
                        for (int i = 0; i < kTcBPT; ++i)
                            lin[i] = 0.f;
                    }
                    if (++k == K) {
                        k = 0;
                        j0 += jnom;
                    }
                }
            }
            // producer and consumers meet between sub-groups (and learn of a failure)
            failed = __syncthreads_or(failed || abort_s);
        }   // sub-groups
        if (failed) {
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                abort_s = 1;
            }
            __syncthreads();
            continue;   // the next fetch sees abort_s and leaves the loop
        }
        // epilogue: combine the kTcQ partial log-sum-exps of each sample
        if (!producer) {
            lse[gh * kTcS + gs] = run_mx;
            lse[(kTcQ + gh) * kTcS + gs] = run_sum;
        }
        __syncthreads();
        if (tid < kTcS && gid[tid] != 0xffffffffu) {
            // the partials combine in float32 (float64 is slow on this part): the largest
            // partial contributes a sum >= 1, so the logarithm is well conditioned.  The
            // template term (thread tid holds sample tid's) is subtracted in float64, so that
            // the difference of two large terms is not rounded to float32.
            float mx = -INFINITY;
            for (int h = 0; h < kTcQ; ++h)
                mx = fmaxf(mx, lse[h * kTcS + tid]);
            float sum = 0.f;
            for (int h = 0; h < kTcQ; ++h) {
                const float m = lse[h * kTcS + tid];
                if (m != -INFINITY)
                    sum += lse[(kTcQ + h) * kTcS + tid] * __expf(m - mx);
            }
            const uint32_t g = gid[tid];
            const double r = (double)mx + (double)__logf(sum) - (kDM ? 0.0 : (double)gqd) - bt.ln_nt;
            if (!kDM && po.q) {
                po.q[g] = gqd;
                po.m[g] = mx;
                po.j[g] = NT - (int)(uint32_t)peak[tid];
            }
            if (!isfinite(r))
                atomicOr(err, kErrNonFinite);
            lnL_tmarg[g] = r;
            if (lnw && lnpw)
                lnw[g] = r + lnpw[g];
        }
        __syncthreads();
    }
    // leave: no bulk copy of this block may still be landing (after a failure the issuer may
    // not have consumed the last windows; bounded wait), no MMA in flight; then free TMEM
    if (warp == kTcStagerWarp && lane == 0)
        for (int b = 0; b < 2; ++b)
            if (phbit(kPhUsed, b))
                tc::mbar_wait(bbar + b, phbit(kPhStg, b) ^ 1u, kWaitNs);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

cudaError_t launch_lnl_tc(const Problem &P, BinTable bt, const double *theta, const uint32_t *perm, int64_t n,
                          double *lnL_tmarg, double *lnL_t, const double *lnpw, double *lnw, int *err,
                          int *tile_counter, cudaStream_t st, const uint32_t *n_dev, int lnl_t_compact,
                          int64_t n_theta, PeakOut po)
{
    if (n_theta <= 0)
        n_theta = n;
    if (n <= 0)
        return cudaSuccess;
    int dev = 0, sms = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!lnl_tc_fits(P, max_smem))
        return cudaErrorInvalidConfiguration;
    const size_t smem = tc_layout(P.K, P.M, P.n_t).end;
    auto kern = P.dist_marg ? lnl_tc_kernel<true> : lnl_tc_kernel<false>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(tile_counter, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    const int64_t tiles = (n + kTcS - 1) / kTcS;
    const int grid = (int)(tiles < sms ? tiles : sms);
    kern<<<grid, kTcThreads, smem, st>>>(P, bt, theta, perm, n, lnL_tmarg, lnL_t, lnpw, lnw, err, tile_counter,
                                          n_dev, n_theta, lnl_t_compact, po);
    return cudaGetLastError();
}

cudaError_t prepare_tc_kernels()
{
    cudaError_t e = allow_max_dynamic_smem(lnl_tc_kernel<false>);
    return e != cudaSuccess ? e : allow_max_dynamic_smem(lnl_tc_kernel<true>);
}

}  // namespace rift
