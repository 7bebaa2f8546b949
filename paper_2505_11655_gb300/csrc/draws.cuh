// Per-sample draws of the sampling priors on the unit cube of prior-CDF coordinates v
// (internal): the product-form histogram and the Gaussian mixture (arXiv:2505.11655
// Sec. II B) and the adaptive-volume cells (Sec. IV A).  Shared by their own draw
// kernels and by the portfolio's, which mixes them (Sec. IV, "Portfolio integrator").
#pragma once

#include "ile_kernels.h"

namespace rift {

// Shared-memory tables of the histogram draw: [6][B+1] running sums, [6][B] reciprocal
// masses, [6][B] log densities (float64 divisions once per block instead of per sample).
__host__ __device__ inline size_t hist_table_doubles(int B) { return 6 * (size_t)(B + 1) + 12 * (size_t)B; }

__device__ __forceinline__ void hist_load_tables(const SamplerDev &S, double *sC)
{
    const int B = S.B;
    double *sR = sC + 6 * (B + 1);
    double *sL = sR + 6 * B;
    for (int e = threadIdx.x; e < 6 * (B + 1); e += blockDim.x)
        sC[e] = S.C[e];
    for (int e = threadIdx.x; e < 6 * B; e += blockDim.x) {
        sR[e] = 1.0 / S.P[e];
        sL[e] = S.L[e];
    }
}

// Draw i of histogram iteration `iter`: Philox4x32-10 (key = seed, counter (i lo, i hi,
// iter, p), p = 0..2; words (0,1) give dimension 2p, (2,3) dimension 2p+1); inverse CDF of
// the piecewise-constant masses.  Writes v, lr = ln p - ln p_s (the distance excluded when
// marginalised) and the six 10-bit bin indices packed (dimension d at bit 10 d).
__device__ __forceinline__ void hist_draw_one(const double *sC, int B, int marg, uint32_t iter, int64_t i,
                                              uint32_t k0, uint32_t k1, double v[6], double &lr, uint64_t &packed)
{
    const double *sR = sC + 6 * (B + 1);
    const double *sL = sR + 6 * B;
    const double inv_b = 1.0 / B;
    // the 53-bit integers m of the uniforms u = m 2^-53
    double m53[6];
#pragma unroll
    for (uint32_t p = 0; p < 3; ++p) {
        U4 r = philox10(U4{(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, p}, k0, k1);
        m53[2 * p] = (double)bits53(r.x, r.y);
        m53[2 * p + 1] = (double)bits53(r.z, r.w);
    }
    lr = 0.0;
    packed = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const double *Cd = sC + d * (B + 1);
        // x = u tot = m (2^-53 tot): both scalings by 2^-53 are exact, so this is the
        // same single rounding as (m 2^-53) tot
        const double x = m53[d] * (Cd[B] * 0x1.0p-53);
        // last b in [0, B-1] with C[b] <= x (C[0] = 0 <= x always).  Non-negative doubles
        // order like their bit patterns read as integers, so the search compares integers
        // (float64 comparisons run on the slow float64 pipe of this part)
        const long long xb = __double_as_longlong(x);
        const long long *Cb = reinterpret_cast<const long long *>(Cd);
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (Cb[mid] <= xb)
                lo = mid;
            else
                hi = mid - 1;
        }
        // t in [0, 1): negative or NaN -> 0, [1, inf] -> the largest double below 1,
        // decided on the bit pattern (integer comparisons)
        long long tb = __double_as_longlong((x - Cd[lo]) * sR[d * B + lo]);
        if (tb < 0 || (tb & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL)
            tb = 0;
        else if (tb >= 0x3ff0000000000000LL)
            tb = 0x3fefffffffffffffLL;
        const double t = __longlong_as_double(tb);
        v[d] = (lo + t) * inv_b;
        if (!(marg && d == 5))
            lr -= sL[d * B + lo];   // ln(B pb / tot), tabulated when the masses change
        packed |= (uint64_t)lo << (10 * d);
    }
}

// The histogram draw's mapping v -> theta.
__device__ __forceinline__ void hist_theta(const double v[6], double d3lo, double d3hi, double th[6])
{
    th[0] = 2.0 * kPi * v[0];
    th[1] = asin(2.0 * v[1] - 1.0);
    th[2] = kPi * v[2];
    th[3] = 2.0 * kPi * v[3];
    th[4] = acos(1.0 - 2.0 * v[4]);
    th[5] = cbrt(d3lo + v[5] * (d3hi - d3lo));
}

// Draw i of AV iteration `iter`: Philox4x32-10 (key = seed, counter (i lo, i hi, iter, p),
// p = 0..3); words 0,1 give the 53-bit integer U of the cell choice cells[floor(U n / 2^53)],
// the next twelve the six in-cell uniforms.  v_d = (coordinate_d + u_d) 2^-level.
__device__ __forceinline__ void av_draw_one(const uint64_t *__restrict__ cells, int64_t n_cells, int level,
                                            uint32_t iter, int64_t i, uint32_t k0, uint32_t k1, double v[6])
{
    const uint64_t mask = level > 0 ? ((1ull << level) - 1ull) : 0ull;
    uint32_t w[16];
#pragma unroll
    for (uint32_t p = 0; p < 4; ++p) {
        const U4 r = philox10(U4{(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, p}, k0, k1);
        w[4 * p] = r.x;
        w[4 * p + 1] = r.y;
        w[4 * p + 2] = r.z;
        w[4 * p + 3] = r.w;
    }
    const uint64_t U = ((uint64_t)(w[0] >> 5) << 26) | (uint64_t)(w[1] >> 6);
    const uint64_t nc = (uint64_t)n_cells;
    const uint64_t c = (__umul64hi(U, nc) << 11) | ((U * nc) >> 53);
    const uint64_t cell = cells[c];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const double u = unit53(w[2 + 2 * d], w[3 + 2 * d]);
        const double coord = (double)((cell >> (level * d)) & mask);
        v[d] = ldexp(__dadd_rn(coord, u), -level);
    }
}

// The AV draw's mapping v -> theta (every operation rounded as written).
__device__ __forceinline__ void av_theta(const double v[6], double d3lo, double d3hi, double th[6])
{
    th[0] = __dmul_rn(2.0 * kPi, v[0]);
    th[1] = asin(__dsub_rn(__dmul_rn(2.0, v[1]), 1.0));
    th[2] = __dmul_rn(kPi, v[2]);
    th[3] = __dmul_rn(2.0 * kPi, v[3]);
    th[4] = acos(__dsub_rn(1.0, __dmul_rn(2.0, v[4])));
    th[5] = cbrt(__dadd_rn(d3lo, __dmul_rn(v[5], __dsub_rn(d3hi, d3lo))));
}

// Key of the level-`level` cell holding v (coordinate d in bits [level d, level (d+1))).
__device__ __forceinline__ uint64_t av_cell_key(const double v[6], int level)
{
    const double side = ldexp(1.0, level);
    uint64_t k = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d)
        k |= (uint64_t)floor(__dmul_rn(v[d], side)) << (level * d);
    return k;
}

// Gaussian-mixture sampling prior: C <= kGmmMax components with weights pi_c and, per
// dimension, a normal of mean mu_cd and width sig_cd truncated to [0, 1].  One iteration's
// draws and densities read a table of kGmmTab doubles built on the host from (pi, mu, sig):
//   [kGmmCum + c]   running sums of pi / sum pi (the component choice)
//   [kGmmK + c]     ln(pi_c / sum pi) - sum_d ln(sig_cd (Phi(b_cd) - Phi(a_cd)) sqrt(2 pi))
//   [kGmmMu + 6c + d], [kGmmSig + ...], [kGmmIsig + ...]   mu, sig, 1 / sig
//   [kGmmPa + ...], [kGmmPd + ...]   Phi(a), Phi(b) - Phi(a), a = -mu/sig, b = (1 - mu)/sig
// and behind them, as float32 (for the float32 modes), K, 1 / sig and mu as a float32 pair
// (hi + lo = mu to ~2^-48).
constexpr int kGmmMax = RIFT_GMM_MAX_COMPONENTS;
constexpr int kGmmCum = 0, kGmmK = kGmmMax, kGmmMu = 2 * kGmmMax, kGmmSig = kGmmMu + 6 * kGmmMax,
              kGmmIsig = kGmmSig + 6 * kGmmMax, kGmmPa = kGmmIsig + 6 * kGmmMax, kGmmPd = kGmmPa + 6 * kGmmMax,
              kGmmF32 = kGmmPd + 6 * kGmmMax;   // float32 section: [C] K, [C][6] 1 / sig, mu hi, mu lo
constexpr int kGmmTab = kGmmF32 + (kGmmMax + 18 * kGmmMax) / 2;
static_assert(kGmmMax % 2 == 0, "the float32 section fills whole doubles");
__host__ __device__ inline float *gmm_kf(double *T) { return reinterpret_cast<float *>(T + kGmmF32); }
__host__ __device__ inline const float *gmm_kf(const double *T) { return reinterpret_cast<const float *>(T + kGmmF32); }
__host__ __device__ inline const float *gmm_isigf(const double *T) { return gmm_kf(T) + kGmmMax; }
__host__ __device__ inline const float *gmm_muhf(const double *T) { return gmm_kf(T) + 7 * kGmmMax; }
__host__ __device__ inline const float *gmm_mulf(const double *T) { return gmm_kf(T) + 13 * kGmmMax; }

// Draw i of GMM iteration `iter`: Philox4x32-10 (key = seed, counter (i lo, i hi, iter, p)):
// p = 8, words 0,1: the 53-bit uniform U of the component, the first c with U < the running
// sum of the weights (the last otherwise); p = 9..11, words (0,1), (2,3): the uniforms u_d;
// v_d = mu + sig Phi^-1(Phi(a) + u_d (Phi(b) - Phi(a))) kept in [0, 1) (every operation
// rounded as written).
__device__ __forceinline__ void gmm_draw_one(const double *T, int C, uint32_t iter, int64_t i, uint32_t k0,
                                             uint32_t k1, double v[6])
{
    const uint32_t lo = (uint32_t)(uint64_t)i, hi = (uint32_t)((uint64_t)i >> 32);
    U4 r = philox10(U4{lo, hi, iter, 8u}, k0, k1);
    const double U = unit53(r.x, r.y);
    int c = C - 1;
    for (int k = 0; k < C - 1; ++k)
        if (U < T[kGmmCum + k]) {
            c = k;
            break;
        }
    double u[6];
#pragma unroll
    for (uint32_t p = 0; p < 3; ++p) {
        r = philox10(U4{lo, hi, iter, 9u + p}, k0, k1);
        u[2 * p] = unit53(r.x, r.y);
        u[2 * p + 1] = unit53(r.z, r.w);
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int e = 6 * c + d;
        const double q = __dadd_rn(T[kGmmPa + e], __dmul_rn(u[d], T[kGmmPd + e]));
        double x = __dadd_rn(T[kGmmMu + e], __dmul_rn(T[kGmmSig + e], normcdfinv(q)));
        if (!(x >= 0.0))
            x = 0.0;
        if (x >= 1.0)
            x = 0x1.fffffffffffffp-1;   // the largest double below 1
        v[d] = x;
    }
}

// The float32 modes' draw: the same uniforms and probability q, the normal quantile in
// float32 on the smaller tail (q or 1 - q, formed in float64), v = mu + sig x in float64.  The
// draw's own density is then evaluated at this v (gmm_ln_density_f32), so the importance
// weight stays consistent; the quantile's few-ulp error moves v by ~1e-7 sig |x|.
__device__ __forceinline__ void gmm_draw_one_f32(const double *T, int C, uint32_t iter, int64_t i, uint32_t k0,
                                                 uint32_t k1, double v[6])
{
    const uint32_t lo = (uint32_t)(uint64_t)i, hi = (uint32_t)((uint64_t)i >> 32);
    U4 r = philox10(U4{lo, hi, iter, 8u}, k0, k1);
    const double U = unit53(r.x, r.y);
    int c = C - 1;
    for (int k = 0; k < C - 1; ++k)
        if (U < T[kGmmCum + k]) {
            c = k;
            break;
        }
    double u[6];
#pragma unroll
    for (uint32_t p = 0; p < 3; ++p) {
        r = philox10(U4{lo, hi, iter, 9u + p}, k0, k1);
        u[2 * p] = unit53(r.x, r.y);
        u[2 * p + 1] = unit53(r.z, r.w);
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int e = 6 * c + d;
        const double q = __dadd_rn(T[kGmmPa + e], __dmul_rn(u[d], T[kGmmPd + e]));
        const float xq = q <= 0.5 ? normcdfinvf((float)q) : -normcdfinvf((float)(1.0 - q));
        double x = fma(T[kGmmSig + e], (double)xq, T[kGmmMu + e]);
        if (!(x >= 0.0))
            x = 0.0;
        if (x >= 1.0)
            x = 0x1.fffffffffffffp-1;
        v[d] = x;
    }
}

// v as a float32 pair (hi + lo = v to ~2^-48; three float64-pipe operations a dimension).
__device__ __forceinline__ void gmm_split(const double v[6], float vh[6], float vl[6])
{
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        vh[d] = (float)v[d];
        vl[d] = (float)(v[d] - (double)vh[d]);
    }
}

// ln(pi_c g_c(v)) of component c in float32: v - mu from the float32 pairs (the difference of
// the high parts is exact when they are close, so z keeps its relative precision even for a
// narrow component), error ~1e-6 in the result.
__device__ __forceinline__ float gmm_ln_comp_f32(const double *T, int c, const float vh[6], const float vl[6])
{
    const float *isf = gmm_isigf(T), *mh = gmm_muhf(T), *ml = gmm_mulf(T);
    float q = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int e = 6 * c + d;
        const float z = ((vh[d] - mh[e]) + (vl[d] - ml[e])) * isf[e];
        q = fmaf(z, z, q);
    }
    return fmaf(-0.5f, q, gmm_kf(T)[c]);
}

__device__ __forceinline__ float gmm_ln_density_f32(const double *T, int C, const float vh[6], const float vl[6])
{
    float mx = -INFINITY, s = 0.f;
    for (int c = 0; c < C; ++c) {
        const float l = gmm_ln_comp_f32(T, c, vh, vl);
        if (l > mx) {
            s = s * __expf(mx - l) + 1.f;
            mx = l;
        } else {
            s += __expf(l - mx);
        }
    }
    return mx + __logf(s);
}

// ln(pi_c g_c(v)) of component c (pi normalised).
__device__ __forceinline__ double gmm_ln_comp(const double *T, int c, const double v[6])
{
    double q = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const double z = (v[d] - T[kGmmMu + 6 * c + d]) * T[kGmmIsig + 6 * c + d];
        q = fma(z, z, q);
    }
    return fma(-0.5, q, T[kGmmK + c]);
}

// ln g(v) of the mixture (running maximum: one exponential per component).
__device__ __forceinline__ double gmm_ln_density(const double *T, int C, const double v[6])
{
    double mx = -INFINITY, s = 0.0;
    for (int c = 0; c < C; ++c) {
        const double l = gmm_ln_comp(T, c, v);
        if (l > mx) {
            s = s * exp(mx - l) + 1.0;
            mx = l;
        } else {
            s += exp(l - mx);
        }
    }
    return mx + log(s);
}

}  // namespace rift
