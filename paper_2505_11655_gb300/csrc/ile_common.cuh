// Shared device-side definitions of the ILE library (internal, not part of the ABI).
//
// Geometry follows arXiv:2505.11655 Sec. II A:
//   source direction n = (cos d cos(a-g), cos d sin(a-g), sin d), arrival delay
//   dt_k = -x_k . n / c; complex response F = F_+ - i F_x; harmonic
//   -2Y_lm(iota, phi_* - phi) with phi_* = 0 (App. conventions, Eq. (hlm));
//   mode coefficient c_k,lm = (D_ref/D) F_k Y_lm.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/rift_ile.h"

namespace rift {

constexpr double kC = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxDet = RIFT_MAX_DET;
constexpr int kMaxModes = RIFT_MAX_MODES;
constexpr int kMaxL = 6;        // largest supported l
constexpr int kMaxWTerms = 5;   // terms of the Wigner-d sum for l <= 6, spin weight -2
constexpr int kMaxPow = 2 * kMaxL + 2;   // largest power of cos(iota/2), sin(iota/2)

// Error flags raised by kernels (OR-ed into a device word).
constexpr int kErrRange = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrTimeout = 4;

// Everything a kernel needs about one problem, passed by value (< 4 KB).
struct Problem {
    int K, M, n_q, n_t;
    int n_q_pad;            // row pitch (floats) of the float32 Q planes
    double fs, t_lo, t_step, gmst, d_ref, kappa;
    // distance marginalisation (dist_marg = 1): x = D_ref/D in [dm_xlo, dm_xhi], prior
    // normalisation ln(3 D_ref^3 / (D_max^3 - D_min^3)), Gauss-Legendre nodes on [-1, 1]
    int dist_marg;
    double dm_xlo, dm_xhi, dm_lnC;
    double dm_lnub;   // dm_lnC + ln((dm_xlo^-3 - dm_xhi^-3) / 3): upper bound offset of the marginal
    double gl16_t[16], gl16_w[16];
    // the float32 quadrature's 10-node rule, as floats (no float64 conversions in the kernels)
    float gl10_tf[10], gl10_wf[10];
    float dm_xlo_f, dm_xhi_f, dm_lnC_f, dm_lnub_f;
    double Dten[kMaxDet][6];   // response tensor: xx, yy, zz, xy, xz, yz
    float Dten_f[kMaxDet][6];  // float copy for the float32 response
    double xpos[kMaxDet][3];   // vertex position / c (seconds)
    double q_t0[kMaxDet];
    // Q-sample position of the first bin: u = ufs0_k + xfs_k . n with n the unit vector
    // to the source (ufs0 = (t_lo - q_t0) fs, xfs = -x fs)
    double ufs0[kMaxDet];
    double xfs[kMaxDet][3];
    int mode_m[kMaxModes];
    // -2Y_lm(iota, .) = sum_t wcoef[t] cos(iota/2)^wpc[t] sin(iota/2)^wps[t]  (normalisation folded in)
    double wcoef[kMaxModes][kMaxWTerms];
    int8_t wpc[kMaxModes][kMaxWTerms];
    int8_t wps[kMaxModes][kMaxWTerms];
    int8_t wn[kMaxModes];
    float wcoef_f[kMaxModes][kMaxWTerms];   // float copy of wcoef
    const double2 *Q64;     // [K][M][n_q]
    const double2 *U64;     // [K][M][M]
    const double2 *V64;
    const float *Qr32;      // [K][2M][n_q_pad] split planes, zero padded
    const float2 *U32;
    const float2 *V32;
    // tensor-core copy of Q: [K][hi, lo][tc_groups][Kp/8][8][8] float16, scaled by 2^e
    // with e from the float bits of max|Q| (*qmax_bits)
    const __half *Qtc;
    int tc_groups;
    // Template term of the tensor-core kernel as a real quadratic form: with z the 2M real
    // components of c_k (re, im per mode), c^H U c + Re c^T V c = z^T T_k z.  Ttc holds
    // T_k^T (= B operand, rows n, K-major) scaled by 2^tt_exp[k], float16 hi/lo:
    // [K][hi, lo][Kp/8 row groups][Kp/8][8][8].
    const __half *Ttc;
    const int *tt_exp;
    const unsigned int *qmax_bits;
};

// ---------------------------------------------------------------- complex helpers
template <typename T> struct Cx { T re, im; };

template <typename T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

__device__ __forceinline__ void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }

// ---------------------------------------------------------------- sky geometry
// Sky trigonometry of one sample, evaluated once in float64.
struct Sky {
    double cd, sd, ch, sh;   // cos/sin of declination and of (alpha - gmst)
};

__device__ __forceinline__ Sky sky_of(double alpha, double delta, double gmst)
{
    Sky s;
    sincos(delta, &s.sd, &s.cd);
    sincos(alpha - gmst, &s.sh, &s.ch);
    return s;
}

// dt_k = -(x_k . n) / c  (x stored already divided by c).
__device__ __forceinline__ double arrival_delay(const Problem &P, int k, const Sky &s)
{
    return -(P.xpos[k][0] * s.cd * s.ch + P.xpos[k][1] * s.cd * s.sh + P.xpos[k][2] * s.sd);
}

// Complex response F = F_+ - i F_x for polarisation psi.  With the sky basis
//   e_a = (-sin h, cos h, 0), e_d = (-sin d cos h, -sin d sin h, cos d)
// and A = e_a.D.e_a, B = e_d.D.e_d, C = e_a.D.e_d, the polarisation frame
// X = -cos psi e_a + sin psi e_d, Y = sin psi e_a + cos psi e_d gives
//   F_+ = cos 2psi (A - B) - 2 sin 2psi C,   F_x = -sin 2psi (A - B) - 2 cos 2psi C,
// i.e. F = (A - B + 2 i C) exp(2 i psi).
template <typename T>
__device__ __forceinline__ Cx<T> response(const Problem &P, int k, const Sky &s, T c2psi, T s2psi)
{
    const double *D = P.Dten[k];
    T ea0 = (T)(-s.sh), ea1 = (T)s.ch;
    T ed0 = (T)(-s.sd * s.ch), ed1 = (T)(-s.sd * s.sh), ed2 = (T)s.cd;
    T xx = (T)D[0], yy = (T)D[1], zz = (T)D[2], xy = (T)D[3], xz = (T)D[4], yz = (T)D[5];
    // D e_a and D e_d
    T da0 = xx * ea0 + xy * ea1, da1 = xy * ea0 + yy * ea1, da2 = xz * ea0 + yz * ea1;
    T dd0 = xx * ed0 + xy * ed1 + xz * ed2;
    T dd1 = xy * ed0 + yy * ed1 + yz * ed2;
    T dd2 = xz * ed0 + yz * ed1 + zz * ed2;
    T A = ea0 * da0 + ea1 * da1;
    T B = ed0 * dd0 + ed1 * dd1 + ed2 * dd2;
    T Cc = ed0 * da0 + ed1 * da1 + ed2 * da2;
    T pr = A - B, pi = (T)2 * Cc;
    return {pr * c2psi - pi * s2psi, pr * s2psi + pi * c2psi};
}

// The same response in float32 from the sky basis vectors already rounded to float
// (ea = (ea0, ea1, 0), ed = (ed0, ed1, ed2)) and the float copy of the tensor; the
// operations are those of response<float>.
__device__ __forceinline__ Cx<float> response_f(const float *D, float ea0, float ea1, float ed0, float ed1, float ed2,
                                                float c2psi, float s2psi)
{
    const float xx = D[0], yy = D[1], zz = D[2], xy = D[3], xz = D[4], yz = D[5];
    const float da0 = xx * ea0 + xy * ea1, da1 = xy * ea0 + yy * ea1, da2 = xz * ea0 + yz * ea1;
    const float dd0 = xx * ed0 + xy * ed1 + xz * ed2;
    const float dd1 = xy * ed0 + yy * ed1 + yz * ed2;
    const float dd2 = xz * ed0 + yz * ed1 + zz * ed2;
    const float A = ea0 * da0 + ea1 * da1;
    const float B = ed0 * dd0 + ed1 * dd1 + ed2 * dd2;
    const float Cc = ed0 * da0 + ed1 * da1 + ed2 * da2;
    const float pr = A - B, pi = 2.f * Cc;
    return {pr * c2psi - pi * s2psi, pr * s2psi + pi * c2psi};
}

// -2Y_lm(iota, -phi) for mode index mi, given powers of cos(iota/2), sin(iota/2).
template <typename T>
__device__ __forceinline__ Cx<T> harmonic(const Problem &P, int mi, const T *cpow, const T *spow, T phi)
{
    T d = 0;
    for (int t = 0; t < P.wn[mi]; ++t)
        d += (T)P.wcoef[mi][t] * cpow[P.wpc[mi][t]] * spow[P.wps[mi][t]];
    T sp, cp;
    sincos_t(-(T)P.mode_m[mi] * phi, &sp, &cp);
    return {d * cp, d * sp};
}

template <typename T>
__device__ __forceinline__ void half_angle_powers(T iota, T *cpow, T *spow)
{
    T sh, ch;
    sincos_t((T)0.5 * iota, &sh, &ch);
    cpow[0] = 1;
    spow[0] = 1;
#pragma unroll
    for (int p = 1; p <= kMaxPow; ++p) {
        cpow[p] = cpow[p - 1] * ch;
        spow[p] = spow[p - 1] * sh;
    }
}

// ---------------------------------------------------------------- counter-based RNG
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// multiplies, key advanced by the Weyl increments between rounds.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = {hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 53-bit uniform in [0, 1) from two words (27 high bits of a, 26 of b).
// the 53-bit integer m of the uniform u = m 2^-53 built from two 32-bit Philox words
__device__ __forceinline__ unsigned long long bits53(uint32_t a, uint32_t b)
{
    return ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
}

__device__ __forceinline__ double unit53(uint32_t a, uint32_t b)
{
    return (double)bits53(a, b) * 0x1.0p-53;
}

// ---------------------------------------------------------------- sort key
// Position of a sample's sky direction along a Hilbert curve over the
// (right ascension, sin declination) square, 2^order cells a side.  Consecutive
// samples in this order stay compact on the sky whatever their density, so a
// tile of consecutive samples has close arrival delays at every detector.
constexpr int kMaxOrder = 10;
constexpr int kMaxCells = 1 << (2 * kMaxOrder);

// Sort key of a sample: which samples share a likelihood tile.  What decides a
// tile's cost is the spread of its samples' arrival delays (the Q window it needs),
// so with one or two detectors the key is built from the delays themselves; with
// three, whose delays lie on a two-dimensional surface, from the sky position.
enum SortMode : int { kSortSky = 0, kSortDelay1 = 1, kSortDelay2 = 2, kSortDelay3 = 3 };

struct SkyGrid {
    int order;     // cells per side = 2^order (kSortDelay3: bits per delay)
    int n_cells;   // 4^order (kSortDelay3: 8^order)
    int mode = kSortSky;
    double gmst = 0.0;
    double x[3][3] = {};   // positions / c of the detectors whose delays form the key (s)
    double span[3] = {};   // |x| / c: those delays lie in [-span, span]
};

__device__ __forceinline__ uint32_t hilbert_index(uint32_t x, uint32_t y, int order)
{
    uint32_t d = 0;
    for (uint32_t s = 1u << (order - 1); s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {   // rotate the quadrant so the curve continues
            if (rx == 1) {
                x = s - 1 - (x & (s - 1));
                y = s - 1 - (y & (s - 1));
            }
            const uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Cell of the (right ascension, sin declination) grid from the prior coordinates
// a = alpha / 2 pi and z = (sin delta + 1) / 2, both in [0, 1).
__device__ __forceinline__ uint32_t sky_cell_v(double a, double z, const SkyGrid &G)
{
    const int side = 1 << G.order;
    const uint32_t x = (uint32_t)min(side - 1, max(0, (int)(a * side)));
    const uint32_t y = (uint32_t)min(side - 1, max(0, (int)(z * side)));
    return hilbert_index(x, y, G.order);
}

__device__ __forceinline__ uint32_t sky_cell(double alpha, double delta, const SkyGrid &G)
{
    if (G.mode != kSortSky) {
        // delays dt_k = -x_k . s with s the unit vector to the source (Earth frame), in
        // float32: the key only orders the samples (at most 2^10 levels per delay; float64
        // transcendentals run on this part's slow float64 pipe)
        float sa, ca, sd, cd;
        sincosf((float)(alpha - G.gmst), &sa, &ca);
        sincosf((float)delta, &sd, &cd);
        const float s0 = cd * ca, s1 = cd * sa, s2 = sd;
        uint32_t q[3];
        const int nd = G.mode == kSortDelay1 ? 1 : G.mode == kSortDelay2 ? 2 : 3;
        const int levels = G.mode == kSortDelay1 ? G.n_cells : (1 << G.order);
        for (int k = 0; k < nd; ++k) {
            const float dt = -((float)G.x[k][0] * s0 + (float)G.x[k][1] * s1 + (float)G.x[k][2] * s2);
            const float u = G.span[k] > 0.0 ? 0.5f * (dt / (float)G.span[k] + 1.0f) : 0.5f;
            q[k] = (uint32_t)min(levels - 1, max(0, (int)(u * (float)levels)));
        }
        if (G.mode == kSortDelay3) {   // Morton interleave of the three quantised delays
            uint32_t key = 0;
            for (int b = 0; b < G.order; ++b)
                for (int k = 0; k < 3; ++k)
                    key |= ((q[k] >> b) & 1u) << (3 * b + k);
            return key;
        }
        return G.mode == kSortDelay1 ? q[0] : hilbert_index(q[0], q[1], G.order);
    }
    const int side = 1 << G.order;
    double a = alpha * (1.0 / (2.0 * kPi));
    a -= floor(a);
    const double z = 0.5 * (sin(delta) + 1.0);
    const uint32_t x = (uint32_t)min(side - 1, max(0, (int)(a * side)));
    const uint32_t y = (uint32_t)min(side - 1, max(0, (int)(z * side)));
    return hilbert_index(x, y, G.order);
}

__device__ __forceinline__ float fn_exp(float x) { return __expf(x); }
__device__ __forceinline__ double fn_exp(double x) { return exp(x); }
__device__ __forceinline__ float fn_log(float x) { return __logf(x); }
// 2^x in float32: one ex2.approx
__device__ __forceinline__ float fn_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double fn_log(double x) { return log(x); }

// ln of the distance-marginal likelihood of one bin.  ln L is exactly a x - b x^2 in
// x = D_ref/D (a, b: data and template terms at D = D_ref); with the prior
// p(D) = 3 D^2 / (D_max^3 - D_min^3) on [D_min, D_max] the marginal is
//   ln( C int x^-4 exp(a x - b x^2) dx ),  x in [D_ref/D_max, D_ref/D_min].
// Composite Gauss-Legendre (NP panels of N nodes) in u = ln x (integrand x^-3 e^{...}, no
// pole), over the part of the range where the exponent is within `thr` of its maximum
// phi_m at x_m: [x_m - d, x_m + d] with d = 2 thr / (g + sqrt(g^2 + 4 b thr)), g the slope
// at x_m (0 for an interior maximum).  The exponent is taken relative to phi_m through
// phi(x) - phi_m = phi'(x_m) (x - x_m) - b (x - x_m)^2, free of cancellation.
// Division where only a placement (a peak, an integration support) depends on it: the
// fast reciprocal-based quotient in float32, the IEEE one in float64.
__device__ __forceinline__ float fn_div(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double fn_div(double x, double y) { return x / y; }

template <typename T, int N, int NP>
__device__ __forceinline__ T ln_dist_marg(const T *gt, const T *gw, T xlo, T xhi, T lnC, T a, T b, T thr)
{
    // the integral is taken relative to the exponent at xm, so xm only has to be close to
    // the maximum
    T xm = b > (T)0 ? fn_div(a, (T)2 * b) : (a > (T)0 ? xhi : xlo);
    xm = xm < xlo ? xlo : (xm > xhi ? xhi : xm);
    const T slope = a - (T)2 * b * xm;
    const T phim = xm * (a - b * xm);
    const T g = slope < (T)0 ? -slope : slope;
    const T den = g + sqrt(g * g + (T)4 * b * thr);
    T L = xlo, R = xhi;
    if (den > (T)0) {
        const T d = fn_div((T)2 * thr, den);
        L = xm - d > xlo ? xm - d : xlo;
        R = xm + d < xhi ? xm + d : xhi;
    }
    const T ul = fn_log(L), h = (fn_log(R) - ul) * ((T)1 / (T)NP);
    // node x = exp(c0 + h t / 2) = exp(c0) exp(h t / 2): the second factor is the same in
    // every panel
    T en[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
        en[i] = fn_exp((T)0.5 * h * gt[i]);
    // panel centre c0 = ln L + (p + 1/2) h: exp(c0) = L e^(h/2) e^(p h), one exponential for
    // all panels
    const T eh = fn_exp((T)0.5 * h), eh2 = eh * eh;
    T ec = L * eh;
    // exponent at node x = ec en_i, u = ln x = c0 + h t_i / 2, dx = x - xm:
    //   slope dx - b dx^2 - 3 u = dx (slope - b dx) + (-3 c0) + (-3 h t_i / 2),
    // the last term once per bin; float32 takes it in base 2 (e^E = 2^(E log2 e)) with log2 e
    // in the coefficients, so that each node costs one ex2
    constexpr bool kF32 = sizeof(T) == 4;
    const T ks = kF32 ? (T)1.4426950408889634 : (T)1;
    const T sl = slope * ks, bs = b * ks;
    T m3h[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
        m3h[i] = (T)-1.5 * ks * h * gt[i];
    T s = (T)0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const T m3c = (T)-3 * ks * (ul + ((T)p + (T)0.5) * h);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const T dx = ec * en[i] - xm;
            const T E = dx * (sl - bs * dx) + (m3c + m3h[i]);
            T e;
            if constexpr (kF32)
                e = fn_exp2(E);
            else
                e = fn_exp(E);
            s += gw[i] * e;
        }
        ec *= eh2;
    }
    return lnC + phim + fn_log((T)0.5 * h * s);
}

// Upper bound of ln_dist_marg: the exponent at its maximum on the range, the x^-3 factor
// integrated over the whole range.
__device__ __forceinline__ float dm_bound32(const Problem &P, float a, float b)
{
    const float xlo = P.dm_xlo_f, xhi = P.dm_xhi_f;
    float xm = b > 0.f ? __fdividef(a, 2.f * b) : (a > 0.f ? xhi : xlo);
    xm = fminf(fmaxf(xm, xlo), xhi);
    return P.dm_lnub_f + xm * (a - b * xm);
}

__device__ __forceinline__ float ln_dist_marg32(const Problem &P, float a, float b)
{
    return ln_dist_marg<float, 10, 2>(P.gl10_tf, P.gl10_wf, P.dm_xlo_f, P.dm_xhi_f, P.dm_lnC_f, a, b, 18.f);
}

__device__ __forceinline__ double ln_dist_marg64(const Problem &P, double a, double b)
{
    return ln_dist_marg<double, 16, 4>(P.gl16_t, P.gl16_w, P.dm_xlo, P.dm_xhi, P.dm_lnC, a, b, 44.0);
}

}  // namespace rift
