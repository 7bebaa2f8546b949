// Portfolio integrator on the device (include/rift_ile.h, rift_ile_portfolio):
// arXiv:2505.11655 Sec. IV, "Portfolio integrator".
//
// The sampling prior is the weighted average of three members' priors on the unit cube
// of prior-CDF coordinates: the product-form histogram (the handle's masses, Sec. II B),
// the adaptive-volume cells (the handle's AV state, Sec. IV A) and a Gaussian mixture
// (Sec. II B's GMM sampler; parameters on the host, a table per iteration on the device).
// One iteration:
//   1. one kernel chooses each draw's member (Philox counter word 3 = 7), draws it with
//      that member's own per-sample draw, and writes ln p - ln p_s of the mixture, the
//      histogram bins of every draw (for the histogram's training) and v (for the
//      others');
//   2. the time-marginalised ln L (the same kernels as every other path), the reduction;
//   3. per-member sums of the weights (online maximum, deterministic block order) give
//      each member's n_ESS, and the GMM's weighted EM sums (per component: S_c and the
//      first two moments, fixed summation order); one copy to the host, where the new
//      weights, the freeze rule and the GMM's new parameters are decided;
//   4. training: the histogram adapts on every sample (the same kernels as
//      rift_ile_adapt); the AV member's own draws are compacted (index order) and go
//      through the AV's live-set, threshold and refinement steps.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "draws.cuh"
#include "ile_handle.h"

using namespace rift;
using namespace rift::host;

namespace {

constexpr int kPfThreads = 256;
constexpr int kPfSumBlocks = 304;
constexpr double kWeightFloor = 0.05;   // no weight below kWeightFloor / N_s
constexpr double kFreezeBelow = 0.05;   // a member under this weight is not trained
constexpr uint32_t kMemberWord = 7;     // Philox counter word 3 of the member choice
constexpr int kNMembers = 3;
constexpr int kSumsGmm = 16;            // offset of the EM sums in PortfolioState::sums
constexpr int kEmStride = 13;           // EM sums per component: S_c, sum r v_d, sum r v_d^2
constexpr double kGmmEps = 0.02;        // pi_c <- (1 - eps) S_c / S + eps / C
constexpr double kGmmSigMin = 1e-3, kGmmSigInit = 0.25;

// Whether `key` is one of the n_cells sorted active cells (binary search).
__device__ __forceinline__ bool in_cells(const uint64_t *__restrict__ cells, int64_t n_cells, uint64_t key)
{
    int64_t lo = 0, hi = n_cells;   // first cell >= key
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cells[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < n_cells && cells[lo] == key;
}

// What one iteration's draw kernel needs to know of the members: bit a of act = member a
// active; multi: more than one active, the member is chosen with thresholds (t0, t1) and
// ln p - ln p_s is the mixture's with weights W; otherwise every draw is member `single`'s.
// lnWf: the float32 modes' ln W_0, ln W_1 - ln V, ln W_2.
struct PfDraw {
    double W[kNMembers];
    double t0, t1;
    float lnWf[kNMembers];
    int act, multi, single, gmm_C;
};

// kF32 (the float32 modes): the mixture's normal quantiles and densities in float32 (the
// draws are then this path's own; the float64 mode keeps every draw and density equal to
// the oracle's to the last bits)
template <bool kF32>
__global__ void __launch_bounds__(kPfThreads) portfolio_draw_kernel(
    SamplerDev S, SkyGrid G, const uint64_t *__restrict__ cells, int64_t n_cells, int level, double lnV,
    double invV, const double *__restrict__ gmm_tab, PfDraw P, uint32_t iter, int64_t n, double *__restrict__ theta,
    double *__restrict__ lnpw, uint64_t *__restrict__ bins, uint32_t *__restrict__ key, double *__restrict__ v_out,
    uint8_t *__restrict__ member)
{
    extern __shared__ double sC[];
    const int B = S.B;
    const bool use_hist = (P.act & 1) != 0, use_av = (P.act & 2) != 0, use_gmm = (P.act & 4) != 0;
    double *sG = sC + (use_hist ? hist_table_doubles(B) : 0);
    if (use_hist)
        hist_load_tables(S, sC);
    if (use_gmm)
        for (int e = threadIdx.x; e < kGmmTab; e += blockDim.x)
            sG[e] = gmm_tab[e];
    __syncthreads();
    const double *sL = sC + 6 * (B + 1) + 6 * B;
    const uint32_t k0 = (uint32_t)S.seed, k1 = (uint32_t)(S.seed >> 32);
    const double d3lo = S.d_min * S.d_min * S.d_min, d3hi = S.d_max * S.d_max * S.d_max;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int m = P.single;
        if (P.multi) {
            const U4 r = philox10(U4{(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, kMemberWord}, k0, k1);
            const double x = unit53(r.x, r.y);
            m = x < P.t0 ? 0 : x < P.t1 ? 1 : 2;
        }
        double v[6], th[6], lr;
        uint64_t packed = 0;
        if (m == 0) {
            hist_draw_one(sC, B, 0, iter, i, k0, k1, v, lr, packed);
            hist_theta(v, d3lo, d3hi, th);
        } else if (m == 1) {
            av_draw_one(cells, n_cells, level, iter, i, k0, k1, v);
            av_theta(v, d3lo, d3hi, th);
            lr = lnV;
        } else if (kF32) {
            gmm_draw_one_f32(sG, P.gmm_C, iter, i, k0, k1, v);
            av_theta(v, d3lo, d3hi, th);
        } else {
            gmm_draw_one(sG, P.gmm_C, iter, i, k0, k1, v);
            av_theta(v, d3lo, d3hi, th);
            lr = -gmm_ln_density(sG, P.gmm_C, v);
        }
        float vh[6], vl[6];
        if (kF32 && use_gmm) {
            gmm_split(v, vh, vl);
            if (m == 2)
                lr = -(double)gmm_ln_density_f32(sG, P.gmm_C, vh, vl);
        }
        if (kF32 && P.multi) {
            // -ln sum_a W_a g_a(v) as a log-sum-exp of ln W_a + ln g_a in float32
            float l0 = -INFINITY, l1 = -INFINITY, l2 = -INFINITY;
            if (use_hist) {
                double lnd = -lr;
                if (m != 0) {
                    lnd = 0.0;
#pragma unroll
                    for (int d = 0; d < 6; ++d) {
                        const int b = min((int)floor(v[d] * (double)B), B - 1);
                        lnd += sL[d * B + b];
                        packed |= (uint64_t)b << (10 * d);
                    }
                }
                l0 = P.lnWf[0] + (float)lnd;
            }
            if (use_av && (m == 1 || in_cells(cells, n_cells, av_cell_key(v, level))))
                l1 = P.lnWf[1];
            if (use_gmm)
                l2 = P.lnWf[2] + (m == 2 ? (float)(-lr) : gmm_ln_density_f32(sG, P.gmm_C, vh, vl));
            const float mx = fmaxf(l0, fmaxf(l1, l2));
            lr = -(double)(mx + __logf(__expf(l0 - mx) + __expf(l1 - mx) + __expf(l2 - mx)));
        } else if (P.multi) {
            // sum over the active members of W_a g_a(v), in member order (each product and
            // sum rounded as written)
            double dens = 0.0;
            if (use_hist) {
                double lnd = -lr;
                if (m != 0) {
                    lnd = 0.0;
#pragma unroll
                    for (int d = 0; d < 6; ++d) {
                        const int b = min((int)floor(v[d] * (double)B), B - 1);
                        lnd += sL[d * B + b];
                        packed |= (uint64_t)b << (10 * d);
                    }
                }
                dens = __dmul_rn(P.W[0], exp(lnd));
            }
            if (use_av && (m == 1 || in_cells(cells, n_cells, av_cell_key(v, level))))
                dens = __dadd_rn(dens, __dmul_rn(P.W[1], invV));
            if (use_gmm)
                dens = __dadd_rn(dens, __dmul_rn(P.W[2], exp(m == 2 ? -lr : gmm_ln_density(sG, P.gmm_C, v))));
            lr = -log(dens);
        }
        double *o = theta + 6 * i;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            o[d] = th[d];
            v_out[6 * i + d] = v[d];
        }
        lnpw[i] = lr;
        bins[i] = packed;
        member[i] = (uint8_t)m;
        // sky-sort key: the histogram draws' as in its own draw kernel, the others' from theta
        key[i] = m == 0 && G.mode == kSortSky ? sky_cell_v(v[0], v[1], G) : sky_cell(th[0], th[1], G);
    }
}

// Running (max, sum exp(x - max), sum exp(2 (x - max)), count) of one member's ln w.
struct MAcc {
    double mx, s1, s2, cnt;
};

__device__ __forceinline__ void macc_add(MAcc &a, double x)
{
    a.cnt += 1.0;
    if (!isfinite(x))
        return;
    if (x > a.mx) {
        const double f = a.mx == -INFINITY ? 0.0 : exp(a.mx - x);
        a.s1 = a.s1 * f + 1.0;
        a.s2 = a.s2 * f * f + 1.0;
        a.mx = x;
    } else {
        const double e = exp(x - a.mx);
        a.s1 += e;
        a.s2 += e * e;
    }
}

__device__ __forceinline__ MAcc macc_merge(MAcc a, MAcc b)
{
    const double mx = fmax(a.mx, b.mx);
    if (mx == -INFINITY)
        return MAcc{mx, 0.0, 0.0, a.cnt + b.cnt};
    const double fa = a.mx == -INFINITY ? 0.0 : exp(a.mx - mx), fb = b.mx == -INFINITY ? 0.0 : exp(b.mx - mx);
    return MAcc{mx, a.s1 * fa + b.s1 * fb, a.s2 * fa * fa + b.s2 * fb * fb, a.cnt + b.cnt};
}

// Pass 1: per block, over a contiguous stripe; partial[blk][member][4].
__global__ void __launch_bounds__(kPfThreads) member_sums_kernel(const double *__restrict__ lnw,
                                                                 const uint8_t *__restrict__ member, int64_t n,
                                                                 double *__restrict__ partial)
{
    __shared__ MAcc sh[kNMembers][kPfThreads];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    MAcc a[kNMembers];
#pragma unroll
    for (int m = 0; m < kNMembers; ++m)
        a[m] = MAcc{-INFINITY, 0.0, 0.0, 0.0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double x = lnw[i];
        const int mi = member[i];
#pragma unroll
        for (int m = 0; m < kNMembers; ++m)   // register-resident accumulators: no dynamic index
            if (mi == m)
                macc_add(a[m], x);
    }
#pragma unroll
    for (int m = 0; m < kNMembers; ++m)
        sh[m][threadIdx.x] = a[m];
    __syncthreads();
    for (int s = kPfThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int m = 0; m < kNMembers; ++m)
                sh[m][threadIdx.x] = macc_merge(sh[m][threadIdx.x], sh[m][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x < kNMembers) {
        const MAcc r = sh[threadIdx.x][0];
        double *o = partial + 4 * kNMembers * blockIdx.x + 4 * threadIdx.x;
        o[0] = r.mx;
        o[1] = r.s1;
        o[2] = r.s2;
        o[3] = r.cnt;
    }
}

// Pass 2: warp m merges member m's partials into out[m][4]: lane l takes blocks l, l + 32,
// ... in order, then the lanes' results merge in a fixed tree (deterministic for a given
// block count; a sequential merge over ~300 blocks is a chain of ~600 float64 exponentials).
__global__ void member_sums_final_kernel(const double *__restrict__ partial, int nb, double *__restrict__ out)
{
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (m >= kNMembers)
        return;
    MAcc a{-INFINITY, 0.0, 0.0, 0.0};
    for (int b = lane; b < nb; b += 32) {
        const double *o = partial + 4 * kNMembers * b + 4 * m;
        a = macc_merge(a, MAcc{o[0], o[1], o[2], o[3]});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const MAcc q{__shfl_down_sync(0xffffffffu, a.mx, o), __shfl_down_sync(0xffffffffu, a.s1, o),
                     __shfl_down_sync(0xffffffffu, a.s2, o), __shfl_down_sync(0xffffffffu, a.cnt, o)};
        if (lane < o)
            a = macc_merge(a, q);
    }
    if (lane == 0) {
        out[4 * m] = a.mx;
        out[4 * m + 1] = a.s1;
        out[4 * m + 2] = a.s2;
        out[4 * m + 3] = a.cnt;
    }
}

// The GMM's weighted EM sums, pass 1.  A block takes a contiguous stripe of samples in
// tiles of kPfThreads: each thread turns one sample into omega_i r_ic (omega_i =
// exp(ln w_i - max ln w), 0 for a non-finite ln w; r_ic = pi_c g_c / sum_c pi_c g_c), then
// thread j < 13 C owns the sum (c, k) = (j / 13, j % 13) of omega r times 1, v_d (k = 1..6)
// or v_d^2 (k = 7..12) and adds the tile's samples to it in index order.  In the float32
// modes the sums are of (v_d - mu_cd) and (v_d - mu_cd)^2 about the component's current
// mean, per tile in float32 and across tiles in float64.  partial[blk][13 C].
template <bool kF32>
__global__ void __launch_bounds__(kPfThreads) gmm_em_partial_kernel(const double *__restrict__ tab, int C,
                                                                    const double *__restrict__ v,
                                                                    const double *__restrict__ lnw, int64_t n,
                                                                    const double *__restrict__ stats, int slot,
                                                                    double *__restrict__ partial)
{
    extern __shared__ double sm[];
    double *sT = sm;                         // [kGmmTab]
    double *sV = sT + kGmmTab;               // [kPfThreads][6]
    double *sW = sV + 6 * kPfThreads;        // [kPfThreads][C]
    // the float32 modes: v as float32 pairs and the weights as float32 in the same bytes
    float *sVh = reinterpret_cast<float *>(sV), *sVl = sVh + 6 * kPfThreads;
    float *sWf = reinterpret_cast<float *>(sW);
    for (int e = threadIdx.x; e < kGmmTab; e += blockDim.x)
        sT[e] = tab[e];
    const double mx = stats[8 * slot + 4];   // max ln w of the batch (finite entries)
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    const int j = threadIdx.x, n_sums = kEmStride * C;
    const int jc = j / kEmStride, jk = j % kEmStride;
    double acc = 0.0;
    __syncthreads();
    for (int64_t t0 = b0; t0 < b1; t0 += kPfThreads) {
        const int64_t i = t0 + threadIdx.x;
        double *w = sW + threadIdx.x * C;
        double *vs = sV + 6 * threadIdx.x;
        if (i < b1) {
            double vi[6];
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                vi[d] = v[6 * i + d];
                if (!kF32)
                    vs[d] = vi[d];
            }
            const double x = lnw[i];
            if (kF32) {
                // the responsibilities and weights in float32 (they only shape the next
                // proposal; its density is evaluated from the parameters it is drawn with)
                const float om = isfinite(x) ? __expf((float)(x - mx)) : 0.f;
                float vh[6], vl[6];
                gmm_split(vi, vh, vl);
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    sVh[6 * threadIdx.x + d] = vh[d];
                    sVl[6 * threadIdx.x + d] = vl[d];
                }
                float lmax = -INFINITY;
                for (int c = 0; c < C; ++c)
                    lmax = fmaxf(lmax, gmm_ln_comp_f32(sT, c, vh, vl));
                float tot = 0.f;
                float *wf = sWf + threadIdx.x * C;
                for (int c = 0; c < C; ++c) {
                    const float e = __expf(gmm_ln_comp_f32(sT, c, vh, vl) - lmax);
                    wf[c] = e;
                    tot += e;
                }
                const float f = om / tot;
                for (int c = 0; c < C; ++c)
                    wf[c] *= f;
            } else {
                const double om = isfinite(x) ? exp(x - mx) : 0.0;
                double lmax = -INFINITY;
                for (int c = 0; c < C; ++c) {
                    w[c] = gmm_ln_comp(sT, c, vi);
                    lmax = fmax(lmax, w[c]);
                }
                double tot = 0.0;
                for (int c = 0; c < C; ++c) {
                    w[c] = exp(w[c] - lmax);
                    tot += w[c];
                }
                const double f = om / tot;
                for (int c = 0; c < C; ++c)
                    w[c] *= f;
            }
        }
        __syncthreads();
        if (kF32 && j < n_sums) {
            // float32 sums over the tile of the moments about the component's current mean
            // (no cancellation for a narrow component), added to the float64 total
            const int cnt = (int)min((int64_t)kPfThreads, b1 - t0);
            float a = 0.f;
            if (jk == 0) {
                for (int q = 0; q < cnt; ++q)
                    a += sWf[q * C + jc];
            } else {
                const int dd = jk <= 6 ? jk - 1 : jk - 7, e = 6 * jc + dd;
                const float mh = gmm_muhf(sT)[e], ml = gmm_mulf(sT)[e];
                for (int q = 0; q < cnt; ++q) {
                    const float z = (sVh[6 * q + dd] - mh) + (sVl[6 * q + dd] - ml);
                    a = fmaf(sWf[q * C + jc], jk <= 6 ? z : z * z, a);
                }
            }
            acc += (double)a;
        } else if (j < n_sums) {
            const int cnt = (int)min((int64_t)kPfThreads, b1 - t0);
            if (jk == 0) {
                for (int q = 0; q < cnt; ++q)
                    acc += sW[q * C + jc];
            } else if (jk <= 6) {
                for (int q = 0; q < cnt; ++q)
                    acc = fma(sW[q * C + jc], sV[6 * q + jk - 1], acc);
            } else {
                for (int q = 0; q < cnt; ++q) {
                    const double x = sV[6 * q + jk - 7];
                    acc = fma(sW[q * C + jc], x * x, acc);
                }
            }
        }
        __syncthreads();
    }
    if (j < n_sums)
        partial[(size_t)blockIdx.x * n_sums + j] = acc;
}

// Pass 2: sum j of the blocks' partials, in block order.
__global__ void gmm_em_final_kernel(const double *__restrict__ partial, int nb, int n_sums, double *__restrict__ out)
{
    for (int j = threadIdx.x; j < n_sums; j += blockDim.x) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b)
            a += partial[(size_t)b * n_sums + j];
        out[j] = a;
    }
}

// flags[i] = draw i is the AV member's; flags[n] = 0
__global__ void av_member_flags_kernel(const uint8_t *__restrict__ member, int64_t n, uint32_t *__restrict__ flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = i < n && member[i] == 1 ? 1u : 0u;
}

__global__ void av_member_compact_kernel(const uint8_t *__restrict__ member, const double *__restrict__ v,
                                         const double *__restrict__ lnL, int64_t n, const uint32_t *__restrict__ rank,
                                         double *__restrict__ v_dst, double *__restrict__ lnL_dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (member[i] != 1)
            continue;
        const int64_t o = rank[i];
#pragma unroll
        for (int d = 0; d < 6; ++d)
            v_dst[6 * o + d] = v[6 * i + d];
        lnL_dst[o] = lnL[i];
    }
}

int grid_n(int64_t n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + kPfThreads - 1) / kPfThreads, cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

// Normalised weights with no active entry below `floor` (water-filling: the entries
// below are set to the floor and the others scaled to fill the rest, until none is below).
void floor_weights(const double in[kNMembers], const int act[kNMembers], double floor, double out[kNMembers])
{
    double tot = 0.0;
    for (int a = 0; a < kNMembers; ++a)
        tot += act[a] ? in[a] : 0.0;
    bool fixed[kNMembers] = {};
    for (int a = 0; a < kNMembers; ++a)
        out[a] = act[a] ? in[a] / tot : 0.0;
    for (;;) {
        bool any = false;
        for (int a = 0; a < kNMembers; ++a)
            if (act[a] && !fixed[a] && out[a] < floor)
                fixed[a] = any = true;
        if (!any)
            return;
        int n_fixed = 0;
        double free_sum = 0.0;
        for (int a = 0; a < kNMembers; ++a) {
            if (fixed[a]) {
                out[a] = floor;
                ++n_fixed;
            } else if (act[a]) {
                free_sum += out[a];
            }
        }
        const double scale = (1.0 - floor * n_fixed) / free_sum;
        for (int a = 0; a < kNMembers; ++a)
            if (act[a] && !fixed[a])
                out[a] *= scale;
    }
}

// ---------------------------------------------------------------- the GMM member (host)

// Standard normal CDF.
double phi_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Initial state: pi = 1/C, sig = 0.25, means on the Kronecker lattice
// mu_cd = frac((c + 1/2) frac(sqrt(p_d))) of the first six primes.
void gmm_init(rift_ile_t::PortfolioState &p, int C)
{
    static const int primes[6] = {2, 3, 5, 7, 11, 13};
    p.gmm_C = C;
    for (int c = 0; c < C; ++c) {
        p.gmm_pi[c] = 1.0 / C;
        for (int d = 0; d < 6; ++d) {
            const double alpha = std::fmod(std::sqrt((double)primes[d]), 1.0);
            p.gmm_mu[6 * c + d] = std::fmod((c + 0.5) * alpha, 1.0);
            p.gmm_sig[6 * c + d] = kGmmSigInit;
        }
    }
}

// The draw and density table of the current parameters (layout in draws.cuh).
void gmm_table(rift_ile_t::PortfolioState &p)
{
    const int C = p.gmm_C;
    std::vector<double> &T = p.gmm_tab_host;
    T.assign(kGmmTab, 0.0);
    double tot = 0.0;
    for (int c = 0; c < C; ++c)
        tot += p.gmm_pi[c];
    double run = 0.0;
    const double ln_sqrt_2pi = 0.5 * std::log(2.0 * M_PI);
    for (int c = 0; c < C; ++c) {
        run += p.gmm_pi[c] / tot;
        T[kGmmCum + c] = run;
        double k = std::log(p.gmm_pi[c] / tot);
        for (int d = 0; d < 6; ++d) {
            const int e = 6 * c + d;
            const double m = p.gmm_mu[e], sg = p.gmm_sig[e];
            const double pa = phi_cdf(-m / sg), pb = phi_cdf((1.0 - m) / sg);
            T[kGmmMu + e] = m;
            T[kGmmSig + e] = sg;
            T[kGmmIsig + e] = 1.0 / sg;
            T[kGmmPa + e] = pa;
            T[kGmmPd + e] = pb - pa;
            k -= std::log(sg) + std::log(pb - pa) + ln_sqrt_2pi;
        }
        T[kGmmK + c] = k;
    }
    float *F = gmm_kf(T.data());
    for (int c = 0; c < C; ++c) {
        F[c] = (float)T[kGmmK + c];
        for (int d = 0; d < 6; ++d) {
            const int e = 6 * c + d;
            const float hi = (float)p.gmm_mu[e];
            F[kGmmMax + e] = (float)(1.0 / p.gmm_sig[e]);
            F[7 * kGmmMax + e] = hi;
            F[13 * kGmmMax + e] = (float)(p.gmm_mu[e] - (double)hi);
        }
    }
}

// One weighted EM step from the sums [C][13] (S_c, sum omega r v_d, sum omega r v_d^2;
// shifted: the last two about the component's current mean).
void gmm_em_apply(rift_ile_t::PortfolioState &p, const double *sums, bool shifted)
{
    const int C = p.gmm_C;
    double S = 0.0;
    for (int c = 0; c < C; ++c)
        S += sums[kEmStride * c];
    if (!(S > 0.0) || !std::isfinite(S))   // no finite ln w: nothing to learn from
        return;
    for (int c = 0; c < C; ++c) {
        const double *q = sums + kEmStride * c;
        const double Sc = q[0];
        const bool live = Sc > 1e-300 * S;
        for (int d = 0; d < 6; ++d) {
            const int e = 6 * c + d;
            double mu = p.gmm_mu[e], var = p.gmm_sig[e] * p.gmm_sig[e];
            if (live && shifted) {
                // the table's float32 pair of the mean, about which the sums were taken
                const double m0 = (double)gmm_muhf(p.gmm_tab_host.data())[e] + (double)gmm_mulf(p.gmm_tab_host.data())[e];
                const double dm = q[1 + d] / Sc;
                mu = m0 + dm;
                var = q[7 + d] / Sc - dm * dm;
            } else if (live) {
                mu = q[1 + d] / Sc;
                var = q[7 + d] / Sc - mu * mu;
            }
            p.gmm_mu[e] = std::min(1.0, std::max(0.0, mu));
            p.gmm_sig[e] = std::min(1.0, std::max(kGmmSigMin, std::sqrt(std::max(var, 0.0))));
        }
        p.gmm_pi[c] = (1.0 - kGmmEps) * Sc / S + kGmmEps / C;
    }
}

int pf_alloc(rift_ile_t *h)
{
    auto &p = h->pf;
    const int64_t N = h->cap;
    int rc;
    if ((rc = dalloc(h, &p.member, (size_t)N)) || (rc = dalloc(h, &p.v, (size_t)N * 6)) ||
        (rc = dalloc(h, &p.v_av, (size_t)N * 6)) || (rc = dalloc(h, &p.lnL_av, (size_t)N)) ||
        (rc = dalloc(h, &p.part, (size_t)4 * kNMembers * kPfSumBlocks)) ||
        (rc = dalloc(h, &p.sums, (size_t)kSumsGmm + kEmStride * kGmmMax)) ||
        (rc = dalloc(h, &p.gmm_part, (size_t)kEmStride * kGmmMax * kPfSumBlocks)) ||
        (rc = dalloc(h, &p.gmm_tab, (size_t)kGmmTab)))
        return rc;
    CK(allow_max_dynamic_smem(portfolio_draw_kernel<false>));
    CK(allow_max_dynamic_smem(portfolio_draw_kernel<true>));
    CK(allow_max_dynamic_smem(gmm_em_partial_kernel<false>));
    CK(allow_max_dynamic_smem(gmm_em_partial_kernel<true>));
    p.alloc = true;
    return RIFT_OK;
}

int pf_restart(rift_ile_t *h, bool with_av, int gmm_components)
{
    auto &p = h->pf;
    p.iter = 0;
    p.have_w = false;
    const int B = h->cfg.n_bins;
    std::vector<double> P0((size_t)6 * B, 1.0 / B);
    CK(cudaMemcpyAsync(h->P, P0.data(), sizeof(double) * 6 * B, cudaMemcpyHostToDevice, h->stream));
    CK(launch_build_cdf(sampler_of(h), h->stream));
    CK(cudaStreamSynchronize(h->stream));   // P0 is a host temporary
    h->launches += 1;
    if (with_av)
        RK(av_restart(h));
    if (gmm_components > 0)
        gmm_init(p, gmm_components);
    else
        p.gmm_C = 0;   // no mixture member since this restart
    return RIFT_OK;
}

int portfolio_iteration(rift_ile_t *h, int64_t n, int slot, bool reset_pooled, const rift_portfolio_config &cfg)
{
    auto &a = h->av;
    auto &p = h->pf;
    cudaStream_t st = h->stream;
    const uint32_t g = p.iter;
    const bool has_av = (cfg.members & RIFT_MEMBER_AV) != 0, has_gmm = (cfg.members & RIFT_MEMBER_GMM) != 0;
    const int act[kNMembers] = {(cfg.members & RIFT_MEMBER_HIST) ? 1 : 0,
                                has_av && (int64_t)g >= cfg.av_start ? 1 : 0,
                                has_gmm && (int64_t)g >= cfg.gmm_start ? 1 : 0};
    const bool joins = (has_av && cfg.av_start > 0 && (int64_t)g == cfg.av_start) ||
                       (has_gmm && cfg.gmm_start > 0 && (int64_t)g == cfg.gmm_start);
    if (!p.have_w || joins) {
        floor_weights(cfg.w_init, act, 0.0, p.W);
        p.have_w = true;
    }
    const int n_act = act[0] + act[1] + act[2];
    double W[kNMembers];
    for (int m = 0; m < kNMembers; ++m)
        W[m] = p.W[m];
    PfDraw P{};
    for (int m = 0; m < kNMembers; ++m)
        P.W[m] = W[m];
    P.t0 = W[0];
    P.t1 = act[2] ? W[0] + W[1] : 2.0;
    P.act = act[0] | (act[1] << 1) | (act[2] << 2);
    P.multi = n_act > 1;
    P.single = act[0] ? 0 : act[1] ? 1 : 2;
    P.gmm_C = p.gmm_C;
    SamplerDev S = sampler_of(h);
    RK(grid_for_batch(h, n));
    // 1. member choice and draws
    CK(mark(h, slot, 0));
    if (act[2]) {
        gmm_table(p);
        CK(cudaMemcpyAsync(p.gmm_tab, p.gmm_tab_host.data(), sizeof(double) * kGmmTab, cudaMemcpyHostToDevice, st));
    }
    const size_t smem = sizeof(double) * ((act[0] ? hist_table_doubles(S.B) : 0) + (act[2] ? kGmmTab : 0));
    const bool f32 = use_fp32(h);
    if (f32) {
        P.lnWf[0] = (float)std::log(W[0]);
        P.lnWf[1] = has_av ? (float)(std::log(W[1]) - std::log(a.V)) : -INFINITY;
        P.lnWf[2] = (float)std::log(W[2]);
    }
    auto draw = f32 ? portfolio_draw_kernel<true> : portfolio_draw_kernel<false>;
    draw<<<grid_n(n), kPfThreads, smem, st>>>(S, h->grid, a.cells, a.n_cells, a.level,
                                              has_av ? std::log(a.V) : 0.0, has_av ? 1.0 / a.V : 0.0, p.gmm_tab, P,
                                              g, n, h->theta, h->lnpw, h->bins, h->key, p.v, p.member);
    CK(cudaGetLastError());
    int sorted = 0;
    if (use_fp32(h))
        CK(launch_sort(h->grid, h->key, n, h->sort_scratch, h->perm, st, &sorted));
    CK(mark(h, slot, 1));
    // 2. likelihood and the iteration's record
    if (!use_fp32(h)) {
        CK(launch_lnl_fp64(h->prob, h->theta, n, h->lnL, nullptr, h->lnpw, h->lnw, h->err, st));
    } else {
        CK(launch_tiled(h, h->theta, n, h->lnL, nullptr, h->lnpw, h->lnw));
        if (h->cfg.precision == RIFT_MIXED)
            RK(refine_batch(h, h->theta, n, h->lnL, h->lnpw, h->lnw));
    }
    CK(mark(h, slot, 2));
    const bool f32_terms = h->cfg.precision == RIFT_FP32;
    CK(launch_reduce(h->lnw, h->lnL, n, h->red_partial, h->stats, slot, h->pooled, reset_pooled ? 1 : 0, h->err, st,
                     f32_terms));
    // 3. per-member n_ESS, the EM sums, the new weights
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kPfSumBlocks, (n + kPfThreads - 1) / kPfThreads));
    member_sums_kernel<<<nb, kPfThreads, 0, st>>>(h->lnw, p.member, n, p.part);
    member_sums_final_kernel<<<1, 32 * kNMembers, 0, st>>>(p.part, nb, p.sums);
    h->launches += 1 + sorted + 1 + 2 + 2;
    const int n_em = act[2] ? kEmStride * p.gmm_C : 0;
    if (act[2]) {
        const size_t em_smem = sizeof(double) * (kGmmTab + 6 * kPfThreads + (size_t)kPfThreads * p.gmm_C);
        auto em = f32 ? gmm_em_partial_kernel<true> : gmm_em_partial_kernel<false>;
        em<<<nb, kPfThreads, em_smem, st>>>(p.gmm_tab, p.gmm_C, p.v, h->lnw, n, h->stats, slot, p.gmm_part);
        gmm_em_final_kernel<<<1, 224, 0, st>>>(p.gmm_part, nb, n_em, p.sums + kSumsGmm);
        CK(cudaGetLastError());
        h->launches += 2;
    }
    double sums[kSumsGmm + kEmStride * kGmmMax];
    CK(cudaMemcpyAsync(sums, p.sums, sizeof(double) * (kSumsGmm + n_em), cudaMemcpyDeviceToHost, st));
    RK(sync_and_err(h));
    double ess[kNMembers];
    int64_t cnt[kNMembers];
    for (int m = 0; m < kNMembers; ++m) {
        cnt[m] = (int64_t)sums[4 * m + 3];
        ess[m] = act[m] && sums[4 * m + 2] > 0.0 ? sums[4 * m + 1] * sums[4 * m + 1] / sums[4 * m + 2] : 0.0;
    }
    double W_next[kNMembers] = {W[0], W[1], W[2]};
    if (cfg.adapt_weights && n_act > 1 && ess[0] + ess[1] + ess[2] > 0.0)
        floor_weights(ess, act, kWeightFloor / n_act, W_next);
    int frozen[kNMembers];
    for (int m = 0; m < kNMembers; ++m)
        frozen[m] = !act[m] || W_next[m] < kFreezeBelow ? 1 : 0;
    // 4. training
    if (!frozen[0]) {
        CK(launch_adapt(S, h->bins, h->lnw, n, h->stats, slot, h->hist_partial, st, f32_terms));
        h->launches += 2;
    }
    if (!frozen[1] && cnt[1] > 0) {
        if (cnt[1] == n) {   // every draw is the AV member's: already in index order
            RK(av_update(h, p.v, h->lnL, n, cfg.p_thr, cfg.n_min_star));
        } else {
            av_member_flags_kernel<<<grid_n(n + 1), kPfThreads, 0, st>>>(p.member, n, a.flags);
            int k = 0;
            CK(launch_scan_u32(a.flags, n + 1, a.scan, st, &k));
            av_member_compact_kernel<<<grid_n(n), kPfThreads, 0, st>>>(p.member, p.v, h->lnL, n, a.flags, p.v_av,
                                                                         p.lnL_av);
            CK(cudaGetLastError());
            h->launches += 2 + k;
            RK(av_update(h, p.v_av, p.lnL_av, cnt[1], cfg.p_thr, cfg.n_min_star));
        }
    }
    if (!frozen[2])
        gmm_em_apply(p, sums + kSumsGmm, f32);
    CK(mark(h, slot, 3));
    for (int m = 0; m < kNMembers; ++m) {
        p.W_last[m] = W[m];
        p.W[m] = W_next[m];
        p.n_ess[m] = ess[m];
        p.n_drawn[m] = cnt[m];
        p.frozen[m] = frozen[m];
        p.active[m] = act[m];
    }
    p.iter += 1;
    return RIFT_OK;
}

}  // namespace

extern "C" {

int rift_ile_portfolio(rift_ile_t *h, int32_t n_iter, int64_t n_per_iter, const rift_portfolio_config *cfg,
                       int32_t restart, rift_ile_result *out)
{
    const int all = RIFT_MEMBER_HIST | RIFT_MEMBER_AV | RIFT_MEMBER_GMM;
    if (!h || !cfg || h->cfg.distance_marg || n_iter < 1 || n_iter > RIFT_MAX_ITER || n_per_iter < 1 ||
        n_per_iter > h->cap || cfg->members < 1 || (cfg->members & ~all) != 0 || cfg->av_start < 0 ||
        cfg->gmm_start < 0 || (cfg->adapt_weights != 0 && cfg->adapt_weights != 1))
        return RIFT_EINVAL;
    const bool has_hist = (cfg->members & RIFT_MEMBER_HIST) != 0, has_av = (cfg->members & RIFT_MEMBER_AV) != 0,
               has_gmm = (cfg->members & RIFT_MEMBER_GMM) != 0;
    if (!has_hist && !(has_av && cfg->av_start == 0) && !(has_gmm && cfg->gmm_start == 0))
        return RIFT_EINVAL;   // no member would draw iteration 0
    for (int m = 0; m < kNMembers; ++m)
        if ((cfg->members >> m) & 1)
            if (!(cfg->w_init[m] > 0.0) || !std::isfinite(cfg->w_init[m]))
                return RIFT_EINVAL;
    if (has_av && (!(cfg->p_thr > 0.0) || !(cfg->p_thr <= 1.0) || cfg->n_min_star < 1 || cfg->capacity < n_per_iter ||
                   cfg->capacity > ((int64_t)1 << 31) - 2 || (h->av.cap != 0 && h->av.cap != cfg->capacity)))
        return RIFT_EINVAL;
    if (has_gmm && (cfg->gmm_components < 1 || cfg->gmm_components > kGmmMax))
        return RIFT_EINVAL;
    const bool fresh = restart != 0 || !h->pf.alloc;
    if (!fresh && (cfg->members != h->pf.members || (has_gmm && h->pf.gmm_C != cfg->gmm_components)))
        return RIFT_EINVAL;   // a change of members or of C needs a restart
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    if (!h->pf.alloc)
        RK(pf_alloc(h));
    if (has_av && h->av.cap == 0) {
        RK(av_alloc(h, cfg->capacity));
        RK(av_restart(h));
    }
    if (fresh) {
        RK(pf_restart(h, has_av, has_gmm ? cfg->gmm_components : 0));
        h->pf.members = cfg->members;
    }
    RK(choose_plan(h, n_per_iter));
    RK(ensure_events(h, n_iter));
    h->timed = true;
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    for (int g = 0; g < n_iter; ++g)
        RK(portfolio_iteration(h, n_per_iter, g, g == 0, *cfg));
    CK(launch_pooled_final(h->pooled, h->final_out, h->iter_dev, 0u, h->stream));
    h->launches += 1;
    h->last_n = n_per_iter;
    return collect_result(h, n_iter, out);
}

int rift_ile_portfolio_info(const rift_ile_t *h, rift_portfolio_info *info)
{
    if (!h || !info)
        return RIFT_EINVAL;
    const auto &p = h->pf;
    std::memset(info, 0, sizeof(*info));
    info->iteration = (int32_t)p.iter;
    for (int m = 0; m < kNMembers; ++m) {
        info->active[m] = p.active[m];
        info->frozen[m] = p.frozen[m];
        info->W_last[m] = p.W_last[m];
        info->W_next[m] = p.W[m];
        info->n_ess[m] = p.n_ess[m];
        info->n_drawn[m] = p.n_drawn[m];
    }
    return RIFT_OK;
}

int rift_ile_portfolio_gmm(const rift_ile_t *h, int32_t capacity, int32_t *n_components, double *pi, double *mu,
                           double *sig)
{
    if (!h)
        return RIFT_EINVAL;
    const auto &p = h->pf;
    if (p.gmm_C == 0)
        return RIFT_ESTATE;
    if (capacity < p.gmm_C)
        return RIFT_EINVAL;
    if (n_components)
        *n_components = p.gmm_C;
    if (pi)
        std::memcpy(pi, p.gmm_pi, sizeof(double) * p.gmm_C);
    if (mu)
        std::memcpy(mu, p.gmm_mu, sizeof(double) * 6 * p.gmm_C);
    if (sig)
        std::memcpy(sig, p.gmm_sig, sizeof(double) * 6 * p.gmm_C);
    return RIFT_OK;
}

}  // extern "C"
