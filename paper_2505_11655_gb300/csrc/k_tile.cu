// Float32 tiled likelihood kernel of the ILE hot path (arXiv:2505.11655 Sec. II A,
// Eq. (def:lnL:Decomposed), time-marginalised on a uniform grid).
//
// Samples arrive sorted by sky cell, so the kTS = 64 samples of a tile need nearly
// the same Q window at every detector.  Per tile:
//   1. prologue (all 256 threads): float64 sky trigonometry and arrival delays,
//      float32 responses F_k and harmonics Y_lm, coefficients c_k,lm = x F_k Y_lm
//      as real components C[s, r] (r = 2m: Re, 2m+1: Im), template term.
//   2. for each chunk of time bins and each detector, on the Q sample grid
//         R[s, c] = sum_r C[s, r] Qr[r, iw0 + c]     (= Re sum_lm conj(c_lm) Q_lm)
//      as a register-blocked 64 x 256 x 2M contraction from shared memory, the
//      next detector's Q window streaming in by cp.async meanwhile; then R is
//      interpolated linearly at every bin's shifted time (interpolation commutes
//      with the mode sum) and summed over detectors;
//   3. the template term is subtracted and each chunk is folded into a per-sample
//      online log-sum-exp; ln L_tmarg = max + ln(sum) - ln n_t in float64.
// Tiles are handed out by an atomic counter (persistent CTAs, one per SM).
#include <cfloat>
#include <cmath>

#include "ile_kernels.h"

namespace rift {

constexpr int kTS = 64;          // samples per tile
constexpr int kNCol = 256;       // Q window columns per chunk
constexpr int kColGroups = kNCol / 32;
constexpr int kTThreads = 256;   // 8 warps
constexpr int kBinsPerLane = 5;  // a chunk holds <= 160 bins
constexpr int kMaxChunkBins = 32 * kBinsPerLane;
constexpr int kPowStride = 16;   // >= kMaxPow + 1
static_assert(kPowStride >= kMaxPow + 1, "power table too short");
// phase B gives every (sample, detector) item its own thread, whole warps per detector
static_assert(kTS * kMaxDet <= kTThreads && kTS % 32 == 0, "one item per thread");

struct TileLayout {
    size_t cs, qb0, qb1, r, bini, binf, sky, par, pw, fx, i0, f0, quad, qpart, gid, end;
};

__host__ __device__ inline size_t al16(size_t o) { return (o + 15) & ~(size_t)15; }

__host__ __device__ inline TileLayout tile_layout(int K, int M, int n_t, bool dbuf)
{
    TileLayout L;
    size_t o = 0;
    L.cs = o;  o = al16(o + (size_t)K * 2 * M * kTS * 4);
    L.qb0 = o; o = al16(o + (size_t)2 * M * kNCol * 4);
    L.qb1 = o; if (dbuf) o = al16(o + (size_t)2 * M * kNCol * 4);
    L.r = o;   o = al16(o + (size_t)kTS * kNCol * 4);
    L.bini = o; o = al16(o + (size_t)n_t * 4);
    L.binf = o; o = al16(o + (size_t)n_t * 4);
    // per-sample tables are sample-minor ([row][kTS]): the lanes of a warp (consecutive
    // samples) touch consecutive words
    L.sky = o; o = al16(o + (size_t)3 * kTS * 8);     // unit vector n to the source (float64)
    L.par = o; o = al16(o + (size_t)9 * kTS * 4);     // c2psi, s2psi, x, phi, and the sky basis e_a, e_d (float32)
    L.pw = o;  o = al16(o + (size_t)2 * kPowStride * kTS * 4);   // cos(i/2)^p, sin(i/2)^p
    L.fx = o;  o = al16(o + (size_t)K * kTS * 8);     // x F_k (float2)
    L.i0 = o;  o = al16(o + (size_t)K * kTS * 4);
    L.f0 = o;  o = al16(o + (size_t)K * kTS * 4);
    L.quad = o; o = al16(o + (size_t)kTS * 4);
    L.qpart = o; o = al16(o + (size_t)4 * kTS * 4);
    L.gid = o; o = al16(o + (size_t)kTS * 4);
    L.end = o;
    return L;
}

static bool tile_dbuf(const Problem &P, int max_smem)
{
    return tile_layout(P.K, P.M, P.n_t, true).end <= (size_t)max_smem;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <bool kDbuf>
__global__ void __launch_bounds__(kTThreads, 1)
lnl_tile_kernel(Problem P, BinTable bt, const double *__restrict__ theta, const uint32_t *__restrict__ perm, int64_t n,
                double *__restrict__ lnL_tmarg, double *__restrict__ lnL_t, const double *__restrict__ lnpw,
                double *__restrict__ lnw, int *err, int *tile_counter, PeakOut po)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int K = P.K, M = P.M, R2 = 2 * M, NT = P.n_t;
    const TileLayout L = tile_layout(K, M, NT, kDbuf);
    float *Cs = reinterpret_cast<float *>(smraw + L.cs);        // [K][2M][kTS]
    float *Qb[2] = {reinterpret_cast<float *>(smraw + L.qb0), reinterpret_cast<float *>(smraw + (kDbuf ? L.qb1 : L.qb0))};
    float *Rs = reinterpret_cast<float *>(smraw + L.r);         // [kTS][kNCol]
    int *bini = reinterpret_cast<int *>(smraw + L.bini);
    float *binf = reinterpret_cast<float *>(smraw + L.binf);
    double *sky = reinterpret_cast<double *>(smraw + L.sky);    // [3][kTS]
    float *par = reinterpret_cast<float *>(smraw + L.par);      // [9][kTS]
    float2 *fx = reinterpret_cast<float2 *>(smraw + L.fx);      // [K][kTS]
    int *i0s = reinterpret_cast<int *>(smraw + L.i0);           // [K][kTS]
    float *f0s = reinterpret_cast<float *>(smraw + L.f0);       // [K][kTS]
    float *qds = reinterpret_cast<float *>(smraw + L.quad);     // [kTS]
    float *qpart = reinterpret_cast<float *>(smraw + L.qpart);  // [4][kTS]
    float *pw = reinterpret_cast<float *>(smraw + L.pw);        // [2 kPowStride][kTS]
    uint32_t *gid = reinterpret_cast<uint32_t *>(smraw + L.gid);
    __shared__ int lo_s[kMaxDet], hi_s[kMaxDet];
    __shared__ int tile_s;
    // bins per chunk for each offset spread that uses the shared window (the float64
    // division once per block: float64 is slow on this part)
    __shared__ int jmax_s[kNCol - 15];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double beta = P.t_step * P.fs;
    const int64_t n_tiles = (n + kTS - 1) / kTS;

    for (int j = tid; j < NT; j += kTThreads) {
        bini[j] = bt.bin_i[j];
        binf[j] = bt.bin_f[j];
    }
    for (int sp = tid; sp <= kNCol - 16; sp += kTThreads) {
        const int jm = !(beta > 0.0) ? kMaxChunkBins : (int)floor((double)(kNCol - 8 - sp - 1) / beta) + 1;
        jmax_s[sp] = max(1, min(jm, kMaxChunkBins));
    }

    for (;;) {
        if (tid == 0)
            tile_s = atomicAdd(tile_counter, 1);
        if (tid < kMaxDet) {
            lo_s[tid] = INT_MAX;
            hi_s[tid] = INT_MIN;
        }
        __syncthreads();
        const int64_t tile = tile_s;
        if (tile >= n_tiles)
            break;

        // ---------------- phase A: per sample, float64 sky trigonometry and scalars
        if (tid < kTS) {
            const int64_t si = tile * kTS + tid;
            uint32_t g = si < n ? perm[si] : 0xffffffffu;
            const bool valid = (int64_t)g < n;
            gid[tid] = valid ? g : 0xffffffffu;
            double th[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
            if (valid)
                for (int d = 0; d < 6; ++d)
                    th[d] = theta[6 * (int64_t)g + d];
            Sky sk = sky_of(th[0], th[1], P.gmst);
            // unit vector to the source in float64 (delays); the sky basis of the response
            // e_a = (-sin h, cos h, 0), e_d = (-sin d cos h, -sin d sin h, cos d) rounded once
            sky[tid] = sk.cd * sk.ch;
            sky[kTS + tid] = sk.cd * sk.sh;
            sky[2 * kTS + tid] = sk.sd;
            float s2p, c2p, shalf, chalf;
            sincosf((float)(2.0 * th[2]), &s2p, &c2p);
            sincosf((float)(0.5 * th[4]), &shalf, &chalf);
            par[tid] = c2p;
            par[kTS + tid] = s2p;
            par[2 * kTS + tid] = valid ? (P.dist_marg ? 1.f : (float)P.d_ref / (float)th[5]) : 0.f;
            par[3 * kTS + tid] = (float)th[3];
            par[4 * kTS + tid] = (float)(-sk.sh);
            par[5 * kTS + tid] = (float)sk.ch;
            par[6 * kTS + tid] = (float)(-sk.sd * sk.ch);
            par[7 * kTS + tid] = (float)(-sk.sd * sk.sh);
            par[8 * kTS + tid] = (float)sk.cd;
            float pc = 1.f, ps = 1.f;
            pw[tid] = 1.f;
            pw[kPowStride * kTS + tid] = 1.f;
            for (int q = 1; q <= kMaxPow; ++q) {
                pc *= chalf;
                ps *= shalf;
                pw[q * kTS + tid] = pc;
                pw[(kPowStride + q) * kTS + tid] = ps;
            }
        }
        __syncthreads();
        // ---------------- phase B: per (sample, detector), delays and x F_k
        for (int it = tid; it < kTS * K; it += kTThreads) {
            const int s = it % kTS, k = it / kTS;
            // Q-sample position of the first bin, (t_lo + dt_k - q_t0_k) fs
            const double u0 =
                fma(P.xfs[k][0], sky[s], fma(P.xfs[k][1], sky[kTS + s], fma(P.xfs[k][2], sky[2 * kTS + s], P.ufs0[k])));
            double fl = floor(u0);
            int i0 = (int)fl;
            i0s[k * kTS + s] = i0;
            f0s[k * kTS + s] = (float)(u0 - fl);
            // offset range at detector k: a warp holds 32 samples of one detector (one item
            // per thread), so reduce over the warp, then one atomic per warp
            const bool valid = gid[s] != 0xffffffffu;
            const int wmin = __reduce_min_sync(0xffffffffu, valid ? i0 : INT_MAX);
            const int wmax = __reduce_max_sync(0xffffffffu, valid ? i0 : INT_MIN);
            if (lane == 0 && wmin != INT_MAX) {
                atomicMin(&lo_s[k], wmin);
                atomicMax(&hi_s[k], wmax);
            }
            const Cx<float> F = response_f(P.Dten_f[k], par[4 * kTS + s], par[5 * kTS + s], par[6 * kTS + s],
                                           par[7 * kTS + s], par[8 * kTS + s], par[s], par[kTS + s]);
            const float amp = par[2 * kTS + s];
            fx[k * kTS + s] = make_float2(amp * F.re, amp * F.im);
        }
        __syncthreads();
        // ---------------- phase C: per (sample, mode), harmonic and coefficients
        for (int it = tid; it < kTS * M; it += kTThreads) {
            const int s = it % kTS, m = it / kTS;
            float d = 0.f;
            for (int t = 0; t < P.wn[m]; ++t)
                d += P.wcoef_f[m][t] * pw[P.wpc[m][t] * kTS + s] * pw[(kPowStride + P.wps[m][t]) * kTS + s];
            float sy, cy;
            sincosf(-(float)P.mode_m[m] * par[3 * kTS + s], &sy, &cy);
            const float yr = d * cy, yi = d * sy;
            for (int k = 0; k < K; ++k) {
                float2 f = fx[k * kTS + s];
                Cs[(k * R2 + 2 * m) * kTS + s] = f.x * yr - f.y * yi;
                Cs[(k * R2 + 2 * m + 1) * kTS + s] = f.x * yi + f.y * yr;
            }
        }
        __syncthreads();
        // ---------------- phase D: template term.  Thread (s, part): sample s = tid % 64,
        // rows a = part, part + 4, ... of every detector, using U^H = U and V^T = V:
        //   c^H U c = sum_a [U_aa |c_a|^2 + 2 Re(conj(c_a) sum_{b>a} U_ab c_b)]
        //   c^T V c = sum_a [V_aa c_a^2   + 2 c_a sum_{b>a} V_ab c_b]
        // The Gram loads are uniform across a warp (one broadcast each).
        {
            const int s = tid & (kTS - 1), part = tid >> 6;
            float acc = 0.f;
            for (int k = 0; k < K; ++k) {
                const float *Ck = Cs + (size_t)k * R2 * kTS + s;
                for (int a = part; a < M; a += 4) {
                    const float2 *Ur = P.U32 + ((size_t)k * M + a) * M;
                    const float2 *Vr = P.V32 + ((size_t)k * M + a) * M;
                    const float ar = Ck[(2 * a) * kTS], ai = Ck[(2 * a + 1) * kTS];
                    float ur = 0.f, ui = 0.f, vr = 0.f, vi = 0.f;
                    for (int b = a + 1; b < M; ++b) {
                        const float cr = Ck[(2 * b) * kTS], ci = Ck[(2 * b + 1) * kTS];
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
            qpart[part * kTS + s] = acc;
        }
        __syncthreads();
        if (tid < kTS)
            qds[tid] = (float)P.kappa * ((qpart[tid] + qpart[kTS + tid]) + (qpart[2 * kTS + tid] + qpart[3 * kTS + tid]));
        __syncthreads();

        int spread = 0;
        for (int k = 0; k < K; ++k)
            spread = max(spread, hi_s[k] - lo_s[k]);
        const bool direct = spread > kNCol - 16;   // no shared window: evaluate from global memory
        const int jmax = direct ? kMaxChunkBins : jmax_s[spread];
        const int n_chunks = (NT + jmax - 1) / jmax;
        const int jnom = (NT + n_chunks - 1) / n_chunks;
        const int n_steps = n_chunks * K;

        // window of step t: detector t % K, bins [j0, j0 + J) of chunk t / K
        auto window = [&](int t, int &iw0, int &ncg) {
            const int k = t % K, j0 = (t / K) * jnom, J = min(jnom, NT - j0);
            const int base = lo_s[k] + bini[j0];
            iw0 = max(base, 0) & ~3;
            (void)J;
            ncg = kColGroups;   // the contraction always covers the full 256-column window
        };
        auto stage = [&](int t, float *dst) {
            int iw0, ncg;
            window(t, iw0, ncg);
            const float *Qk = P.Qr32 + (size_t)(t % K) * R2 * P.n_q_pad + iw0;
            const int per_row = ncg * 8;
            for (int e = tid; e < R2 * per_row; e += kTThreads) {
                const int r = e / per_row, c4 = e - r * per_row;
                cp_async16(dst + r * kNCol + 4 * c4, Qk + (size_t)r * P.n_q_pad + 4 * c4);
            }
            cp_async_commit();
        };

        if (!direct) {
            if (tid == 0 && lo_s[0] + bini[0] < 0)
                atomicOr(err, kErrRange);
            stage(0, Qb[0]);
        }

        // running log-sum-exp per sample over the bins of the data term alone (the template
        // term enters once, in the epilogue) and the bin of its maximum
        float run_mx[8], run_sum[8];
        int run_j[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            run_mx[p] = -INFINITY;
            run_sum[p] = 0.f;
            run_j[p] = 0;
        }
        float lin[8][kBinsPerLane];
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
            for (int q = 0; q < kBinsPerLane; ++q)
                lin[p][q] = 0.f;

        for (int t = 0; t < n_steps; ++t) {
            const int k = t % K, j0 = (t / K) * jnom, J = min(jnom, NT - j0);
            const int *i0k = i0s + k * kTS;
            const float *f0k = f0s + k * kTS;
            if (!direct) {
                int iw0, ncg;
                window(t, iw0, ncg);
                cp_async_wait_all();
                __syncthreads();   // window t visible; every thread is past step t-1
                if (kDbuf && t + 1 < n_steps)
                    stage(t + 1, Qb[(t + 1) & 1]);
                const float *Q = Qb[kDbuf ? (t & 1) : 0];
                // thread (warp, lane): samples warp*8 .. +8, columns 4 lane + 128 g + v
                float acc[8][8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        acc[i][c] = 0.f;
                const float *Ck = Cs + (size_t)k * R2 * kTS + warp * 8;
                const float *Ql = Q + 4 * lane;
                // operands of step r + 1 are loaded while step r's 64 FMAs issue
                float4 na0 = *reinterpret_cast<const float4 *>(Ck);
                float4 na1 = *reinterpret_cast<const float4 *>(Ck + 4);
                float4 nb0 = *reinterpret_cast<const float4 *>(Ql);
                float4 nb1 = *reinterpret_cast<const float4 *>(Ql + 128);
                for (int r = 0; r < R2; ++r) {
                    const float a[8] = {na0.x, na0.y, na0.z, na0.w, na1.x, na1.y, na1.z, na1.w};
                    const float b[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};
                    const int rn = r + 1 < R2 ? r + 1 : r;
                    na0 = *reinterpret_cast<const float4 *>(Ck + rn * kTS);
                    na1 = *reinterpret_cast<const float4 *>(Ck + rn * kTS + 4);
                    nb0 = *reinterpret_cast<const float4 *>(Ql + rn * kNCol);
                    nb1 = *reinterpret_cast<const float4 *>(Ql + rn * kNCol + 128);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            acc[i][c] = fmaf(a[i], b[c], acc[i][c]);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float *Rrow = Rs + (warp * 8 + i) * kNCol + 4 * lane;
                    *reinterpret_cast<float4 *>(Rrow) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                    *reinterpret_cast<float4 *>(Rrow + 128) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
                }
                __syncthreads();   // R complete (and, single-buffered, the Q window consumed)
                if (!kDbuf && t + 1 < n_steps)
                    stage(t + 1, Qb[0]);
                int bi[kBinsPerLane];
                float bf[kBinsPerLane];
#pragma unroll
                for (int q = 0; q < kBinsPerLane; ++q) {
                    const int jj = min(lane + 32 * q, J - 1);
                    bi[q] = bini[j0 + jj];
                    bf[q] = binf[j0 + jj];
                }
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int s = warp + 8 * p;
                    const bool ok = gid[s] != 0xffffffffu;
                    // padding samples use the tile's lowest offset, which keeps every read in the row
                    const float *Rrow = Rs + s * kNCol + ((ok ? i0k[s] : lo_s[k]) - iw0);
                    const float f0 = ok ? f0k[s] : 0.f;
#pragma unroll
                    for (int q = 0; q < kBinsPerLane; ++q) {
                        const float sf = f0 + bf[q];
                        const int carry = sf >= 1.f;
                        const float fr = sf - (float)carry;
                        const float *rr = Rrow + bi[q] + carry;
                        const float r0 = rr[0], r1 = rr[1];
                        lin[p][q] += fmaf(fr, r1 - r0, r0);
                    }
                }
            } else {
                const float *Qk = P.Qr32 + (size_t)k * R2 * P.n_q_pad;
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int s = warp + 8 * p;
                    if (gid[s] == 0xffffffffu)
                        continue;
                    const int i0 = i0k[s];
                    const float f0 = f0k[s];
#pragma unroll
                    for (int q = 0; q < kBinsPerLane; ++q) {
                        const int jj = lane + 32 * q;
                        if (jj < J) {
                            const float sf = f0 + binf[j0 + jj];
                            const int carry = sf >= 1.f;
                            const float fr = sf - (float)carry;
                            const int c = i0 + bini[j0 + jj] + carry;
                            if (c < 0 || c + 1 >= P.n_q) {
                                atomicOr(err, kErrRange);
                                continue;
                            }
                            float v = 0.f;
                            for (int r = 0; r < R2; ++r) {
                                const float *row = Qk + (size_t)r * P.n_q_pad + c;
                                const float q0 = __ldg(row), q1 = __ldg(row + 1);
                                v = fmaf(Cs[(k * R2 + r) * kTS + s], fmaf(fr, q1 - q0, q0), v);
                            }
                            lin[p][q] += v;
                        }
                    }
                }
            }
            if (k == K - 1) {
                // fold the chunk's bins into each sample's running log-sum-exp; the
                // eight samples' warp reductions are interleaved
                float cmx[8], cs[8];
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const float qd = qds[warp + 8 * p];
                    cmx[p] = -INFINITY;
                    if (P.dist_marg) {
                        // distance marginal per bin: upper bounds first; the sample's bin with
                        // the highest bound is evaluated (by the lane holding it), and bins
                        // whose bound lies more than 40 below the larger of that value and
                        // the running maximum cannot move the marginal (< e^-40): left out
                        float bnd[kBinsPerLane], bl = -INFINITY, al = 0.f;
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q) {
                            bnd[q] = lane + 32 * q < J ? dm_bound32(P, lin[p][q], qd) : -INFINITY;
                            if (bnd[q] > bl) {
                                bl = bnd[q];
                                al = lin[p][q];
                            }
                        }
                        float bmax = bl;
#pragma unroll
                        for (int o = 16; o; o >>= 1)
                            bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
                        const int owner = __ffs(__ballot_sync(0xffffffffu, bl == bmax)) - 1;
                        float vbest = -INFINITY;
                        if (lane == owner && bmax > -INFINITY)
                            vbest = ln_dist_marg32(P, al, qd);
                        vbest = __shfl_sync(0xffffffffu, vbest, owner);
                        const float thr = lnL_t ? -INFINITY : fmaxf(run_mx[p], vbest) - 40.f;
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q) {
                            lin[p][q] = (lane + 32 * q < J && bnd[q] >= thr) ? ln_dist_marg32(P, lin[p][q], qd)
                                                                              : -INFINITY;
                            if (lane + 32 * q < J)
                                cmx[p] = fmaxf(cmx[p], lin[p][q]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q)
                            if (lane + 32 * q < J)
                                cmx[p] = fmaxf(cmx[p], lin[p][q]);
                    }
                }
                if (lnL_t) {
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        const uint32_t g = gid[warp + 8 * p];
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q)
                            if (lane + 32 * q < J && g != 0xffffffffu)
                                lnL_t[(int64_t)g * NT + j0 + lane + 32 * q] =
                                    P.dist_marg ? (double)lin[p][q] : (double)lin[p][q] - (double)qds[warp + 8 * p];
                    }
                }
#pragma unroll
                for (int o = 16; o; o >>= 1)
#pragma unroll
                    for (int p = 0; p < 8; ++p)
                        cmx[p] = fmaxf(cmx[p], __shfl_xor_sync(0xffffffffu, cmx[p], o));
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    if (cmx[p] > run_mx[p]) {
                        // a new running maximum (warp-uniform): its bin, the lowest holding it
                        int jc = INT_MAX;
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q)
                            if (lane + 32 * q < J && lin[p][q] == cmx[p])
                                jc = min(jc, j0 + lane + 32 * q);
                        run_j[p] = __reduce_min_sync(0xffffffffu, jc);
                    }
                    cmx[p] = fmaxf(run_mx[p], cmx[p]);
                    cs[p] = 0.f;
#pragma unroll
                    for (int q = 0; q < kBinsPerLane; ++q) {
                        if (lane + 32 * q < J)
                            cs[p] += __expf(lin[p][q] - cmx[p]);
                        lin[p][q] = 0.f;
                    }
                }
#pragma unroll
                for (int o = 16; o; o >>= 1)
#pragma unroll
                    for (int p = 0; p < 8; ++p)
                        cs[p] += __shfl_xor_sync(0xffffffffu, cs[p], o);
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    run_sum[p] = (run_mx[p] == -INFINITY ? 0.f : run_sum[p] * __expf(run_mx[p] - cmx[p])) + cs[p];
                    run_mx[p] = cmx[p];
                }
            }
        }
        // ---------------- epilogue: lane p writes sample warp + 8 p
        if (lane < 8) {
            float mxv = run_mx[0], smv = run_sum[0];
            int jv = run_j[0];
#pragma unroll
            for (int p = 1; p < 8; ++p)
                if (lane == p) {
                    mxv = run_mx[p];
                    smv = run_sum[p];
                    jv = run_j[p];
                }
            const int s = warp + 8 * lane;
            const uint32_t g = gid[s];
            if (g != 0xffffffffu) {
                // the log-sum-exp in float32 like the partials (smv >= 1); the template term
                // subtracted in float64, so that the difference of two large terms is not
                // rounded to float32
                const double r =
                    (double)mxv + (double)__logf(smv) - (P.dist_marg ? 0.0 : (double)qds[s]) - bt.ln_nt;
                if (!P.dist_marg && po.q) {
                    po.q[g] = qds[s];
                    po.m[g] = mxv;
                    po.j[g] = jv;
                }
                if (!isfinite(r))
                    atomicOr(err, kErrNonFinite);
                lnL_tmarg[g] = r;
                if (lnw && lnpw)
                    lnw[g] = r + lnpw[g];
            }
        }
        __syncthreads();
    }
}

size_t lnl_fp32_smem_bytes(const Problem &P)
{
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return tile_layout(P.K, P.M, P.n_t, tile_dbuf(P, max_smem)).end;
}

cudaError_t launch_lnl_fp32(const Problem &P, BinTable bt, const double *theta, const uint32_t *perm, int64_t n,
                            double *lnL_tmarg, double *lnL_t, const double *lnpw, double *lnw, int *err,
                            int *tile_counter, cudaStream_t st, PeakOut po)
{
    if (n <= 0)
        return cudaSuccess;
    int dev = 0, sms = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool dbuf = tile_dbuf(P, max_smem);
    const size_t smem = tile_layout(P.K, P.M, P.n_t, dbuf).end;
    if (smem > (size_t)max_smem)
        return cudaErrorInvalidConfiguration;
    auto kern = dbuf ? lnl_tile_kernel<true> : lnl_tile_kernel<false>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(tile_counter, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    const int64_t tiles = (n + kTS - 1) / kTS;
    const int grid = (int)(tiles < sms ? tiles : sms);
    kern<<<grid, kTThreads, smem, st>>>(P, bt, theta, perm, n, lnL_tmarg, lnL_t, lnpw, lnw, err, tile_counter, po);
    return cudaGetLastError();
}

cudaError_t prepare_tile_kernels()
{
    cudaError_t e = allow_max_dynamic_smem(lnl_tile_kernel<true>);
    return e != cudaSuccess ? e : allow_max_dynamic_smem(lnl_tile_kernel<false>);
}

}  // namespace rift
