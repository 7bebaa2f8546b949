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
constexpr int kTcThreads = kTcConsumers + 32;   // plus one producer warp: TMA staging and MMA issue
constexpr int kTcProducerWarp = kTcConsumers / 32;
constexpr int kTcQ = kTcConsumers / kTcS;  // threads per sample in the gather (bin quarters)
constexpr int kTcBPT = 16;         // bins per thread per chunk
constexpr int kTcMaxBins = kTcQ * kTcBPT;
// R is kept transposed, Rt[column][sample]: the drain (lane = sample, fixed column) and
// the gather (lane = sample, per-sample column) both touch bank = sample, conflict-free.
constexpr int kTcPow = 16;
constexpr uint64_t kWaitNs = 1000000000ull;
// A tile whose samples span more than this many Q samples at some detector is cut
// into contiguous sub-groups (compact along the sort order) that are windowed apart.
constexpr int kTcSpreadLimit = 64;

struct TcLayout {
    size_t a, b, r, bini, binf, i0, f0, inv, quad, gid, lse, bar, tptr, end;
    size_t sky, par, pw, fx, qpart;   // prologue scratch, aliased on the B buffers
    int kp;
};

__host__ __device__ inline size_t tc_al(size_t o, size_t a = 128) { return (o + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int K, int M, int n_t)
{
    TcLayout L;
    L.kp = (2 * M + 15) / 16 * 16;
    size_t o = 0;
    L.a = o;
    o = tc_al(o + (size_t)K * 2 * kTcS * L.kp * 2);
    L.b = o;
    const size_t bbytes = (size_t)2 * 2 * kTcW * L.kp * 2;
    size_t s = L.b;
    L.sky = s;   s = tc_al(s + (size_t)kTcS * 4 * 8, 16);
    L.par = s;   s = tc_al(s + (size_t)kTcS * 8 * 4, 16);
    L.pw = s;    s = tc_al(s + (size_t)kTcS * 2 * kTcPow * 4, 16);
    L.fx = s;    s = tc_al(s + (size_t)K * kTcS * 8, 16);
    L.qpart = s; s = tc_al(s + (size_t)kTcQ * kTcS * 4, 16);
    o = tc_al(L.b + (bbytes > s - L.b ? bbytes : s - L.b));
    L.r = o;
    const size_t rbytes = (size_t)kTcW * kTcS * 4, cbytes = (size_t)K * 2 * M * kTcS * 4;
    o = tc_al(o + (rbytes > cbytes ? rbytes : cbytes), 16);
    L.bini = o; o = tc_al(o + (size_t)n_t * 4, 16);
    L.binf = o; o = tc_al(o + (size_t)n_t * 4, 16);
    L.i0 = o;   o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.f0 = o;   o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.inv = o;  o = tc_al(o + (size_t)K * kTcS * 4, 16);
    L.quad = o; o = tc_al(o + (size_t)kTcS * 4, 16);
    L.gid = o;  o = tc_al(o + (size_t)kTcS * 4, 16);
    L.lse = o;  o = tc_al(o + (size_t)2 * kTcQ * kTcS * 4, 16);
    L.bar = o;  o = tc_al(o + 6 * 8, 16);
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

// ---------------------------------------------------------------- the kernel

// kDM: distance marginalisation (a separate instantiation, so that the plain path keeps
// its registers)
template <bool kDM>
__global__ void __launch_bounds__(kTcThreads, 1)
lnl_tc_kernel(Problem P, BinTable bt, const double *__restrict__ theta, const uint32_t *__restrict__ perm, int64_t n,
              double *__restrict__ lnL_tmarg, double *__restrict__ lnL_t, const double *__restrict__ lnpw,
              double *__restrict__ lnw, int *err, int *tile_counter)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int K = P.K, M = P.M, R2 = 2 * M, NT = P.n_t;
    const TcLayout L = tc_layout(K, M, NT);
    const int kp = L.kp, kcores = kp / 8;
    __half *As = reinterpret_cast<__half *>(sm + L.a);          // [K][2][kTcS x kp] canonical K-major
    __half *Bs = reinterpret_cast<__half *>(sm + L.b);          // [2 buf][2 part][kTcW x kp]
    float *Rs = reinterpret_cast<float *>(sm + L.r);            // Rt [kTcW][kTcS] (prologue: C [K][2M][kTcS])
    int *bini = reinterpret_cast<int *>(sm + L.bini);
    float *binf = reinterpret_cast<float *>(sm + L.binf);
    int *i0s = reinterpret_cast<int *>(sm + L.i0);              // [K][kTcS]
    float *f0s = reinterpret_cast<float *>(sm + L.f0);
    float *invs = reinterpret_cast<float *>(sm + L.inv);        // [K][kTcS] 2^-(row exponent + Q exponent)
    float *qds = reinterpret_cast<float *>(sm + L.quad);
    uint32_t *gid = reinterpret_cast<uint32_t *>(sm + L.gid);
    uint64_t *bbar = reinterpret_cast<uint64_t *>(sm + L.bar);  // [0,1] windows staged
    uint64_t *fullb = bbar + 2;   // [0,1] MMAs of an accumulator complete (tcgen05.commit)
    uint64_t *emptyb = bbar + 4;  // [0,1] accumulator drained by the 16 consumer warps
    uint32_t *tptr = reinterpret_cast<uint32_t *>(sm + L.tptr);
    double *sky = reinterpret_cast<double *>(sm + L.sky);
    float *par = reinterpret_cast<float *>(sm + L.par);
    float *pw = reinterpret_cast<float *>(sm + L.pw);
    float2 *fx = reinterpret_cast<float2 *>(sm + L.fx);
    float *qpart = reinterpret_cast<float *>(sm + L.qpart);
    float *lse = reinterpret_cast<float *>(sm + L.lse);         // [2][kTcQ][kTcS] running max, sum
    float *Cs = Rs;
    __shared__ int lo_s[kMaxDet], hi_s[kMaxDet];        // current sub-group's offset range
    __shared__ int glo[kTcS][kMaxDet], ghi[kTcS][kMaxDet], gstart[kTcS + 1];
    __shared__ int tile_s, abort_s, ngroups_s;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double beta = P.t_step * P.fs;
    const int64_t n_tiles = (n + kTcS - 1) / kTcS;
    const uint32_t idesc = tc::idesc_f16_f32(kTcS, kTcW);
    const uint32_t sbo = (uint32_t)kcores * 128u;
    const size_t part_halves = (size_t)kTcW * kp;                 // one B part
    const uint32_t part_bytes = (uint32_t)(part_halves * 2);
    const int qexp = q_exponent(*P.qmax_bits);

    for (int j = tid; j < NT; j += blockDim.x) {
        bini[j] = bt.bin_i[j];
        binf[j] = bt.bin_f[j];
    }
    if (warp == 0)
        tc::tmem_alloc(tptr, 256);
    if (tid == 0) {
        for (int i = 0; i < 4; ++i)
            tc::mbar_init(bbar + i, 1);
        for (int i = 4; i < 6; ++i)
            tc::mbar_init(bbar + i, kTcConsumers / 32);
        tc::fence_mbar_init();
        abort_s = 0;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tptr;
    // completed-phase counters per buffer: windows staged (producer), MMA commits
    // (producer and consumers keep their own copies), accumulator drains (producer)
    uint32_t nstage[2] = {0u, 0u}, ncommit[2] = {0u, 0u}, nfull[2] = {0u, 0u}, ndrain[2] = {0u, 0u};
    const bool producer = warp == kTcProducerWarp;

    for (;;) {
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

        // ---------------- prologue A: sky trigonometry (float64) and per-sample scalars
        if (tid < kTcS) {
            const int64_t si = tile * kTcS + tid;
            uint32_t g = si < n ? perm[si] : 0xffffffffu;
            const bool valid = (int64_t)g < n;
            gid[tid] = valid ? g : 0xffffffffu;
            double th[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
            if (valid)
                for (int d = 0; d < 6; ++d)
                    th[d] = theta[6 * (int64_t)g + d];
            Sky sk = sky_of(th[0], th[1], P.gmst);
            double *sp = sky + 4 * tid;
            sp[0] = sk.cd;
            sp[1] = sk.sd;
            sp[2] = sk.ch;
            sp[3] = sk.sh;
            float s2p, c2p, shalf, chalf;
            sincosf((float)(2.0 * th[2]), &s2p, &c2p);
            sincosf((float)(0.5 * th[4]), &shalf, &chalf);
            float *pp = par + 8 * tid;
            pp[0] = c2p;
            pp[1] = s2p;
            pp[2] = valid ? (kDM ? 1.f : (float)(P.d_ref / th[5])) : 0.f;
            pp[3] = (float)th[3];
            float *pc = pw + tid * 2 * kTcPow, *ps = pc + kTcPow;
            pc[0] = 1.f;
            ps[0] = 1.f;
            for (int q = 1; q <= kMaxPow; ++q) {
                pc[q] = pc[q - 1] * chalf;
                ps[q] = ps[q - 1] * shalf;
            }
        }
        __syncthreads();
        // ---------------- B: delays, interpolation node split, x F_k
        for (int it = tid; tid < kTcConsumers && it < kTcS * K; it += kTcConsumers) {
            const int s = it % kTcS, k = it / kTcS;
            const double *sp = sky + 4 * s;
            Sky sk{sp[0], sp[1], sp[2], sp[3]};
            const float *pp = par + 8 * s;
            double u0 = (P.t_lo + arrival_delay(P, k, sk) - P.q_t0[k]) * P.fs;
            double fl = floor(u0);
            int i0 = (int)fl;
            i0s[k * kTcS + s] = i0;
            f0s[k * kTcS + s] = (float)(u0 - fl);
            if (gid[s] != 0xffffffffu) {
                atomicMin(&lo_s[k], i0);
                atomicMax(&hi_s[k], i0);
            }
            Cx<float> F = response<float>(P, k, sk, pp[0], pp[1]);
            fx[k * kTcS + s] = make_float2(pp[2] * F.re, pp[2] * F.im);
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
        // ---------------- C: harmonics and coefficients C [K][2M][kTcS] (float32)
        for (int it = tid; tid < kTcConsumers && it < kTcS * M; it += kTcConsumers) {
            const int s = it % kTcS, m = it / kTcS;
            const float *pc = pw + s * 2 * kTcPow, *ps = pc + kTcPow;
            float d = 0.f;
            for (int t = 0; t < P.wn[m]; ++t)
                d += (float)P.wcoef[m][t] * pc[P.wpc[m][t]] * ps[P.wps[m][t]];
            float sy, cy;
            sincosf(-(float)P.mode_m[m] * par[8 * s + 3], &sy, &cy);
            const float yr = d * cy, yi = d * sy;
            for (int k = 0; k < K; ++k) {
                float2 f = fx[k * kTcS + s];
                Cs[(k * R2 + 2 * m) * kTcS + s] = f.x * yr - f.y * yi;
                Cs[(k * R2 + 2 * m + 1) * kTcS + s] = f.x * yi + f.y * yr;
            }
        }
        __syncthreads();
        // ---------------- D: template term (Hermitian U, symmetric V halving), kTcQ threads per sample
        if (tid < kTcConsumers) {
            const int s = tid & (kTcS - 1), part = tid >> 7;
            float acc = 0.f;
            for (int k = 0; k < K; ++k) {
                const float *Ck = Cs + (size_t)k * R2 * kTcS + s;
                for (int a = part; a < M; a += kTcQ) {
                    const float2 *Ur = P.U32 + ((size_t)k * M + a) * M;
                    const float2 *Vr = P.V32 + ((size_t)k * M + a) * M;
                    const float ar = Ck[(2 * a) * kTcS], ai = Ck[(2 * a + 1) * kTcS];
                    float ur = 0.f, ui = 0.f, vr = 0.f, vi = 0.f;
                    for (int b = a + 1; b < M; ++b) {
                        const float cr = Ck[(2 * b) * kTcS], ci = Ck[(2 * b + 1) * kTcS];
                        const float2 u = __ldg(Ur + b), v = __ldg(Vr + b);
                        ur = fmaf(u.x, cr, fmaf(-u.y, ci, ur));
                        ui = fmaf(u.x, ci, fmaf(u.y, cr, ui));
                        vr = fmaf(v.x, cr, fmaf(-v.y, ci, vr));
                        vi = fmaf(v.x, ci, fmaf(v.y, cr, vi));
                    }
                    const float2 ud = __ldg(Ur + a), vd = __ldg(Vr + a);
                    const float a2r = ar * ar - ai * ai, a2i = 2.f * ar * ai;
                    acc += ud.x * (ar * ar + ai * ai) + 2.f * (ar * ur + ai * ui);
                    acc += (vd.x * a2r - vd.y * a2i) + 2.f * (ar * vr - ai * vi);
                }
            }
            qpart[part * kTcS + s] = acc;
        }
        __syncthreads();
        if (tid < kTcS)
            qds[tid] = (float)P.kappa * ((qpart[tid] + qpart[kTcS + tid]) + (qpart[2 * kTcS + tid] + qpart[3 * kTcS + tid]));

        // ---------------- E: A operand, float16 hi/lo with a power-of-two scale per (sample, detector)
        {
            for (int it = tid; tid < kTcConsumers && it < kTcS * K; it += kTcConsumers) {
                const int s = it % kTcS, k = it / kTcS;
                const float *Ck = Cs + (size_t)k * R2 * kTcS + s;
                float mx = 0.f;
                for (int r = 0; r < R2; ++r)
                    mx = fmaxf(mx, fabsf(Ck[r * kTcS]));
                int ex = 0;
                if (mx > 0.f)
                    frexpf(mx, &ex);
                const int es = mx > 0.f ? 14 - ex : 0;
                const float sc = ldexpf(1.f, es);
                invs[k * kTcS + s] = ldexpf(1.f, -es - qexp);
                __half *Ahi = As + (size_t)(k * 2) * kTcS * kp;
                __half *Alo = Ahi + (size_t)kTcS * kp;
                const int rowbase = ((s >> 3) * kcores * 8 + (s & 7)) * 8;
                for (int r = 0; r < kp; ++r) {
                    const float v = r < R2 ? Ck[r * kTcS] * sc : 0.f;
                    const __half hi = __float2half_rn(v);
                    const __half lo = __float2half_rn(v - __half2float(hi));
                    const int off = rowbase + (r >> 3) * 64 + (r & 7);
                    Ahi[off] = hi;
                    Alo[off] = lo;
                }
            }
            tc::fence_proxy_async_smem();
        }
        __syncthreads();

        // gather / fold ownership: thread -> sample s, bin quarter h of every chunk
        const int gs = tid & (kTcS - 1), gh = (tid >> 7) & (kTcQ - 1);
        const bool gok = !producer && gid[gs] != 0xffffffffu;
        const float gqd = qds[gs];
        float run_mx = -INFINITY, run_sum = 0.f;
        int failed = 0;
        const int ngroups = ngroups_s;
        for (int grp = 0; grp < ngroups && !failed; ++grp) {
            int glo_k[kMaxDet];
            int spread = 0;
            for (int k = 0; k < K; ++k) {
                glo_k[k] = glo[grp][k];
                spread = max(spread, ghi[grp][k] - glo[grp][k]);
            }
            const bool in_grp = gs >= gstart[grp] && gs < gstart[grp + 1];
            int jmax = !(beta > 0.0) ? kTcMaxBins : (int)floor((double)(kTcW - 11 - spread) / beta) + 1;
            jmax = max(1, min(jmax, kTcMaxBins));
            const int n_chunks = (NT + jmax - 1) / jmax;
            const int jnom = (NT + n_chunks - 1) / n_chunks;
            const int n_steps = n_chunks * K;
            // window of step t: detector t % K, bins of chunk t / K; clamped so that a
            // window never leaves the allocation of the Q copy
            auto win0 = [&](int t) {
                const int k = t % K, j0 = (t / K) * jnom;
                return min(max(glo_k[k] + bini[j0], 0), 8 * (P.tc_groups - 16)) & ~7;
            };

            if (producer) {
                // ============ producer warp, lane 0: stage windows, issue MMAs
                if (lane == 0) {
                    auto stage = [&](int t) {
                        const int k = t % K, b = t & 1;
                        const int g0 = win0(t) >> 3;
                        const __half *src = P.Qtc + ((size_t)k * 2 * P.tc_groups + g0) * (size_t)kp * 8;
                        __half *dst = Bs + (size_t)b * 2 * part_halves;
                        tc::mbar_expect_tx(bbar + b, 2 * part_bytes);
                        tc::bulk_g2s(dst, src, part_bytes, bbar + b);
                        tc::bulk_g2s(dst + part_halves, src + (size_t)P.tc_groups * kp * 8, part_bytes, bbar + b);
                        ++nstage[b];
                    };
                    stage(0);
                    if (n_steps > 1)
                        stage(1);
                    for (int t = 0; t < n_steps && !failed; ++t) {
                        const int k = t % K, b = t & 1;
                        // window t staged; accumulator b drained by the consumers
                        if (!tc::mbar_wait(bbar + b, (nstage[b] - 1) & 1u, kWaitNs) ||
                            (ncommit[b] > ndrain[b] && !tc::mbar_wait(emptyb + b, ndrain[b] & 1u, kWaitNs))) {
                            failed = 1;
                            break;
                        }
                        if (ncommit[b] > ndrain[b])
                            ++ndrain[b];
                        tc::tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(b * kTcW);
                        const uint32_t a_hi = tc::smem_u32(As + (size_t)(k * 2) * kTcS * kp);
                        const uint32_t a_lo = a_hi + (uint32_t)(kTcS * kp * 2);
                        const uint32_t b_hi = tc::smem_u32(Bs + (size_t)b * 2 * part_halves);
                        const uint32_t b_lo = b_hi + part_bytes;
                        for (int kk = 0; kk < kp / 16; ++kk) {
                            const uint32_t o = (uint32_t)kk * 256u;
                            tc::mma_f16(d, tc::smem_desc(a_hi + o, 128, sbo), tc::smem_desc(b_hi + o, 128, sbo), idesc,
                                        kk > 0);
                            tc::mma_f16(d, tc::smem_desc(a_hi + o, 128, sbo), tc::smem_desc(b_lo + o, 128, sbo), idesc, 1);
                            tc::mma_f16(d, tc::smem_desc(a_lo + o, 128, sbo), tc::smem_desc(b_hi + o, 128, sbo), idesc, 1);
                        }
                        tc::mma_commit(fullb + b);
                        ++ncommit[b];
                        // window t + 1 goes into the other buffer once the MMAs of step t - 1 are done
                        if (t >= 1 && t + 1 < n_steps) {
                            const int bo = (t - 1) & 1;
                            if (!tc::mbar_wait(fullb + bo, (ncommit[bo] - 1) & 1u, kWaitNs)) {
                                failed = 1;
                                break;
                            }
                            stage(t + 1);
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
                for (int t = 0; t < n_steps; ++t) {
                    const int k = t % K, b = t & 1, j0 = (t / K) * jnom, J = min(jnom, NT - j0);
                    const int jq = (J + kTcQ - 1) / kTcQ;                 // bins per quarter
                    const int jb = j0 + gh * jq, jn = max(0, min(jq, j0 + J - jb));   // this thread's bins
                    // one lane per warp waits for the MMAs of step t
                    int ok = 1;
                    if (lane == 0)
                        ok = tc::mbar_wait(fullb + b, nfull[b] & 1u, kWaitNs) ? 1 : 0;
                    ++nfull[b];
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    tc::tc_fence_after();
                    // The rows of sample quarter q (TMEM lanes 32q..) are drained and gathered by
                    // the same four warps (warp & 3 == q), so each quarter synchronises on its own
                    // barrier: its warps are past their previous gather (its rows of R are free);
                    // agree on failure.
                    const int qbar = 2 + (warp & 3);
                    if (tc::named_bar_or(qbar, kTcConsumers / 4, !ok || abort_s)) {
                        failed = 1;
                        break;
                    }
                    {
                        // drain accumulator b: warp quarter q = rows 32q.., column block w / 4 of 32
                        const int q = warp & 3, cb = warp >> 2;
                        float *Rcol = Rs + (32 * cb) * kTcS + 32 * q + lane;
                        uint32_t v[32];
                        tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTcW + 32 * cb), v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            Rcol[i * kTcS] = __uint_as_float(v[i]);
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        tc::mbar_arrive(emptyb + b);
                    tc::named_bar(qbar, kTcConsumers / 4);   // this quarter's rows of R complete
                    const int iw0 = win0(t);
                    // padding samples and samples of other sub-groups read at the group's lowest
                    // offset, which keeps every read in the row; their sums are discarded
                    const bool mine = gok && in_grp;
                    const float *Rcol = Rs + ((mine ? i0s[k * kTcS + gs] : glo_k[k]) - iw0) * kTcS + gs;
                    const float ff = mine ? f0s[k * kTcS + gs] : 0.f;
                    const float sc = invs[k * kTcS + gs];
                    if (k == 0) {
                        // this thread's bins of the chunk, shared by every detector (idle slots
                        // re-read the chunk's last bin)
#pragma unroll
                        for (int i = 0; i < kTcBPT; ++i) {
                            const int j = min(jb + i, j0 + J - 1);
                            bj[i] = bini[j];
                            bfj[i] = binf[j];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < kTcBPT; ++i) {
                        const float sf = ff + bfj[i];
                        const int carry = sf >= 1.f;
                        const float fr = sf - (float)carry;
                        const float *rr = Rcol + (bj[i] + carry) * kTcS;
                        const float r0 = rr[0], r1 = rr[kTcS];
                        lin[i] = fmaf(sc, fmaf(fr, r1 - r0, r0), lin[i]);
                    }
                    if (k == K - 1) {
                        // fold this thread's bins of the chunk into its running log-sum-exp
                        float cmx = -INFINITY;
                        if (kDM) {
                            // distance marginal per bin: a cheap upper bound first; the bin
                            // with the highest bound is evaluated, and a bin whose bound lies
                            // more than 40 below the larger of that value and the running
                            // maximum cannot move the marginal (< e^-40): left out
                            float bnd[kTcBPT], bmax = -INFINITY, abest = 0.f;
#pragma unroll
                            for (int i = 0; i < kTcBPT; ++i) {
                                bnd[i] = i < jn ? dm_bound32(P, lin[i], gqd) : -INFINITY;
                                if (bnd[i] > bmax) {
                                    bmax = bnd[i];
                                    abest = lin[i];
                                }
                            }
                            const float vbest = jn > 0 ? ln_dist_marg32(P, abest, gqd) : -INFINITY;
                            // (every bin exact when the per-bin values are written out)
                            const float thr = lnL_t ? -INFINITY : fmaxf(run_mx, vbest) - 40.f;
#pragma unroll
                            for (int i = 0; i < kTcBPT; ++i) {
                                lin[i] = (i < jn && bnd[i] >= thr) ? ln_dist_marg32(P, lin[i], gqd) : -INFINITY;
                                if (i < jn)
                                    cmx = fmaxf(cmx, lin[i]);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < kTcBPT; ++i) {
                                lin[i] -= gqd;
                                if (i < jn)
                                    cmx = fmaxf(cmx, lin[i]);
                            }
                        }
                        if (lnL_t && gok && in_grp) {
                            for (int i = 0; i < jn; ++i)
#pragma unroll
                                for (int u = 0; u < kTcBPT; ++u)
                                    if (u == i)
                                        lnL_t[(int64_t)gid[gs] * NT + jb + i] = (double)lin[u];
                        }
                        if (jn > 0 && in_grp) {
                            const float nm = fmaxf(run_mx, cmx);
                            float cs = 0.f;
#pragma unroll
                            for (int i = 0; i < kTcBPT; ++i)
                                if (i < jn)
                                    cs += __expf(lin[i] - nm);
                            run_sum = (run_mx == -INFINITY ? 0.f : run_sum * __expf(run_mx - nm)) + cs;
                            run_mx = nm;
                        }
#pragma unroll
                        for (int i = 0; i < kTcBPT; ++i)
                            lin[i] = 0.f;
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
            float mx = -INFINITY;
            for (int h = 0; h < kTcQ; ++h)
                mx = fmaxf(mx, lse[h * kTcS + tid]);
            double sum = 0.0;
            for (int h = 0; h < kTcQ; ++h) {
                const float m = lse[h * kTcS + tid];
                if (m != -INFINITY)
                    sum += (double)lse[(kTcQ + h) * kTcS + tid] * exp((double)m - (double)mx);
            }
            const uint32_t g = gid[tid];
            double r = (double)mx + log(sum) - log((double)NT);
            if (!isfinite(r))
                atomicOr(err, kErrNonFinite);
            lnL_tmarg[g] = r;
            if (lnw && lnpw)
                lnw[g] = r + lnpw[g];
        }
        __syncthreads();
    }
    // leave: make sure no bulk copy or MMA of this block is still in flight, then free TMEM
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 256);
    }
}

cudaError_t launch_lnl_tc(const Problem &P, BinTable bt, const double *theta, const uint32_t *perm, int64_t n,
                          double *lnL_tmarg, double *lnL_t, const double *lnpw, double *lnw, int *err,
                          int *tile_counter, cudaStream_t st)
{
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
    kern<<<grid, kTcThreads, smem, st>>>(P, bt, theta, perm, n, lnL_tmarg, lnL_t, lnpw, lnw, err,
                                                  tile_counter);
    return cudaGetLastError();
}

cudaError_t prepare_tc_kernels()
{
    cudaError_t e = allow_max_dynamic_smem(lnl_tc_kernel<false>);
    return e != cudaSuccess ? e : allow_max_dynamic_smem(lnl_tc_kernel<true>);
}

}  // namespace rift
