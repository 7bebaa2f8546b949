/*
 * Plain FP64 CPU oracle for the extrinsic-marginalised likelihood integral
 * (ILE) of arXiv:2505.11655 ("Narrowing RIFT").
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg call this code to produce expected values; the product
 * (the CUDA library) never links, loads or calls it, and shares no code,
 * header, table or constant generator with it.
 *
 * Written for obviousness, not speed: one extrinsic sample at a time, every
 * step in the order the paper states it, in double precision.  The only
 * parallelism is an OpenMP loop over independent samples.
 *
 * Sections followed:
 *   strain and modes ............ Sec. II A, Eqs. (strain), (strain_mode)
 *   L-frame harmonic angles ..... App. (waveform conventions), Eq. (hlm), phi_* = 0
 *   detector response, delay .... Sec. II A (F_k = F_+ - i F_x, t_k = t_c - x_k . n)
 *   decomposed ln L ............. Sec. II A, Eq. (def:lnL:Decomposed)
 *   Monte Carlo marginal ........ Sec. II B, Eq. (lnL:MonteCarlo)
 *   adaptive Cartesian sampler .. Sec. II B (product-form p_s, 1-D marginals)
 *   n_eff ....................... Sec. II C, Eq. (neff)
 *   n_ESS ....................... Sec. IV A (adaptive volume), Kish form
 *   time marginalisation ........ App. (timing): every evaluation is time marginalised
 * Readings where the paper is silent are listed beside each function.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C_SI 299792458.0
#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t n_det;
    const double *det_tensor; /* [K][3][3] */
    const double *det_pos;    /* [K][3], metres */
    double gmst;              /* Greenwich sidereal angle (rad) */
    int32_t n_modes;
    const int32_t *lm;        /* [M][2] */
    double fs;                /* Q sample rate (Hz) */
    int32_t n_q;
    const double *q_t0;       /* [K] time of Q sample 0 (s) */
    const double *Q;          /* [K][M][n_q] complex128, interleaved */
    const double *U;          /* [K][M][M] complex128 */
    const double *V;          /* [K][M][M] complex128 */
    double t_lo, t_hi;
    int32_t n_t;
    double d_ref, d_min, d_max;
    double kappa;             /* 1/4 as printed in Eq. (def:lnL:Decomposed) */
    int32_t dist_marg;        /* 1: ln L marginalised over the distance prior (see orc_ln_dist_marg) */
} orc_problem;

/* ---------------------------------------------------------------- geometry */

/* Unit vector toward the source in the Earth-fixed frame; alpha is right
 * ascension, delta declination, g the Greenwich sidereal angle. */
static void orc_source_dir(double alpha, double delta, double g, double s[3])
{
    s[0] = cos(delta) * cos(alpha - g);
    s[1] = cos(delta) * sin(alpha - g);
    s[2] = sin(delta);
}

/* Arrival time at detector k relative to the geocentre: t_k - t_c = -x_k . n / c
 * (Sec. II A), n read as the unit vector toward the source. */
double orc_delay(const double x[3], double alpha, double delta, double g)
{
    double s[3];
    orc_source_dir(alpha, delta, g, s);
    return -(x[0] * s[0] + x[1] * s[1] + x[2] * s[2]) / ORC_C_SI;
}

static double orc_quadform(const double *D, const double a[3], const double b[3])
{
    double r = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            r += a[i] * D[3 * i + j] * b[j];
    return r;
}

/* Detector response F_+ and F_x for response tensor D (Anderson et al. 2001,
 * PRD 63 042003, App. B, written in the sky basis):
 *   e_a = (-sin(a-g), cos(a-g), 0), e_d = (-sin d cos(a-g), -sin d sin(a-g), cos d)
 *   X = -cos psi e_a + sin psi e_d,  Y = sin psi e_a + cos psi e_d
 *   F_+ = X.D.X - Y.D.Y,  F_x = X.D.Y + Y.D.X
 * The paper combines them as F = F_+ - i F_x (Sec. II A).  psi enters only here. */
void orc_antenna(const double *D, double alpha, double delta, double psi, double g,
                 double *fplus, double *fcross)
{
    double h = alpha - g;
    double ea[3] = {-sin(h), cos(h), 0.0};
    double ed[3] = {-sin(delta) * cos(h), -sin(delta) * sin(h), cos(delta)};
    double X[3], Y[3];
    for (int i = 0; i < 3; ++i) {
        X[i] = -cos(psi) * ea[i] + sin(psi) * ed[i];
        Y[i] = sin(psi) * ea[i] + cos(psi) * ed[i];
    }
    *fplus = orc_quadform(D, X, X) - orc_quadform(D, Y, Y);
    *fcross = orc_quadform(D, X, Y) + orc_quadform(D, Y, X);
}

static double orc_fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i)
        r *= i;
    return r;
}

/* Wigner-d factor of the spin-weight -2 harmonic (the closed-form sum of
 * Ajith et al. 2007, LIGO-T070017):
 *   d = sum_k (-1)^k sqrt((l+m)!(l-m)!(l+2)!(l-2)!) / ((l+m-k)!(l-2-k)! k! (k+2-m)!)
 *         cos(i/2)^(2l+m-2-2k) sin(i/2)^(2k+2-m),  k = max(0, m-2) .. min(l+m, l-2). */
double orc_wigner_d(int l, int m, double iota)
{
    double c = cos(0.5 * iota), s = sin(0.5 * iota);
    int k0 = m - 2 > 0 ? m - 2 : 0;
    int k1 = (l + m < l - 2) ? l + m : l - 2;
    double pre = sqrt(orc_fact(l + m) * orc_fact(l - m) * orc_fact(l + 2) * orc_fact(l - 2));
    double d = 0.0;
    for (int k = k0; k <= k1; ++k) {
        double term = pre / (orc_fact(l + m - k) * orc_fact(l - 2 - k) * orc_fact(k) * orc_fact(k + 2 - m));
        term *= pow(c, 2 * l + m - 2 - 2 * k) * pow(s, 2 * k + 2 - m);
        d += (k % 2) ? -term : term;
    }
    return d;
}

/* Spin-weighted harmonic -2Y_lm(theta, varphi) = sqrt((2l+1)/4pi) d e^{i m varphi}. */
double complex orc_sYlm(int l, int m, double theta, double varphi)
{
    return sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI)) * orc_wigner_d(l, m, theta) * cexp(I * m * varphi);
}

/* Per-sample mode coefficients c_k,lm = (D_ref/D) F_k Y_lm and delays dt_k.
 * theta = (alpha, delta, psi, phi, iota, D).  The harmonic is evaluated at
 * (iota, phi_* - phi) with phi_* = 0 (Eq. (hlm)). */
void orc_coeffs(const orc_problem *P, const double *theta, double complex *F, double complex *Ylm,
                double complex *c, double *dt)
{
    double alpha = theta[0], delta = theta[1], psi = theta[2], phi = theta[3], iota = theta[4];
    double x = P->d_ref / theta[5];
    for (int m = 0; m < P->n_modes; ++m)
        Ylm[m] = orc_sYlm(P->lm[2 * m], P->lm[2 * m + 1], iota, -phi);
    for (int k = 0; k < P->n_det; ++k) {
        double fp, fx;
        orc_antenna(P->det_tensor + 9 * k, alpha, delta, psi, P->gmst, &fp, &fx);
        F[k] = fp - I * fx;
        dt[k] = orc_delay(P->det_pos + 3 * k, alpha, delta, P->gmst);
        for (int m = 0; m < P->n_modes; ++m)
            c[k * P->n_modes + m] = x * F[k] * Ylm[m];
    }
}

static double complex orc_cget(const double *base, int64_t idx)
{
    return base[2 * idx] + I * base[2 * idx + 1];
}

/* Quadratic (template) term of Eq. (def:lnL:Decomposed):
 *   kappa sum_k [ sum conj(c_lm) U_k,lm,l'm' c_l'm' + Re sum c_lm V_k,lm,l'm' c_l'm' ]
 * which equals the printed |F|^2 Y* Y' U + Re(F^2 Y Y' V) form with c = x F Y.
 * The V term carries Re as in the summed form (the matrix form's missing Re is
 * read as a typesetting slip). */
double orc_quad(const orc_problem *P, const double complex *c)
{
    int M = P->n_modes;
    double total = 0.0;
    for (int k = 0; k < P->n_det; ++k) {
        const double complex *ck = c + k * M;
        double complex su = 0.0, sv = 0.0;
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) {
                su += conj(ck[a]) * orc_cget(P->U, ((int64_t)k * M + a) * M + b) * ck[b];
                sv += ck[a] * orc_cget(P->V, ((int64_t)k * M + a) * M + b) * ck[b];
            }
        total += creal(su) + creal(sv);
    }
    return P->kappa * total;
}

/* Time bin j of the marginalisation grid: inclusive, evenly spaced (t_lo..t_hi). */
double orc_bin_time(const orc_problem *P, int j)
{
    if (P->n_t == 1)
        return P->t_lo;
    return P->t_lo + j * (P->t_hi - P->t_lo) / (P->n_t - 1);
}

/* Data term at one bin: Re sum_k sum_lm conj(c_k,lm) Q_k,lm(t_j + dt_k), with Q
 * linearly interpolated between its samples, real and imaginary parts alike.
 * Returns 0 on success, -1 if an interpolation node falls outside the Q window
 * (an error, never a clamp). */
int orc_data_term(const orc_problem *P, const double complex *c, const double *dt, int j, double *out)
{
    int M = P->n_modes;
    double lin = 0.0;
    double tj = orc_bin_time(P, j);
    for (int k = 0; k < P->n_det; ++k) {
        double u = (tj + dt[k] - P->q_t0[k]) * P->fs;
        double fl = floor(u);
        if (!(fl >= 0.0) || fl + 1.0 > (double)(P->n_q - 1))
            return -1;
        int64_t i = (int64_t)fl;
        double f = u - fl;
        for (int m = 0; m < M; ++m) {
            int64_t base = ((int64_t)k * M + m) * P->n_q;
            double complex q = (1.0 - f) * orc_cget(P->Q, base + i) + f * orc_cget(P->Q, base + i + 1);
            lin += creal(conj(c[k * M + m]) * q);
        }
    }
    *out = lin;
    return 0;
}

/* ln L at every bin and its time marginal
 *   ln L_tmarg = ln( (1/N_t) sum_j exp(ln L_j) ),
 * a Riemann mean over the inclusive grid (uniform time prior on the window).
 * lnL_t may be NULL.  Returns 0 or -1 (Q window exceeded). */
/* ---------------------------------------------------------------- distance marginal */

/* 16-point Gauss-Legendre nodes and weights on [-1, 1], set once by the Python side
 * (a library routine) before any evaluation. */
static double orc_gl_t[16], orc_gl_w[16];

void orc_set_gauss_legendre16(const double *t, const double *w)
{
    for (int i = 0; i < 16; ++i) {
        orc_gl_t[i] = t[i];
        orc_gl_w[i] = w[i];
    }
}

/* Distance-marginal likelihood of one bin.  ln L is exactly a x - b x^2 in x = D_ref/D
 * (a: data term at D = D_ref, b: template term at D = D_ref).  With the prior
 * p(D) = 3 D^2 / (D_max^3 - D_min^3) on [D_min, D_max],
 *   ln int p(D) exp(a x - b x^2) dD = ln( 3 D_ref^3 / (D_max^3 - D_min^3) int x^-4 e^{a x - b x^2} dx )
 * over x in [D_ref/D_max, D_ref/D_min].  Evaluated by composite 16-point Gauss-Legendre
 * in u = ln x (integrand x^-3 e^{a x - b x^2}) with 200 equal panels over the part of the
 * interval where a x - b x^2 is within 80 of its maximum on the interval (outside it the
 * integrand is below e^-80 times the peak even with the x^-3 factor).  That part is
 * [x_m - d, x_m + d] with x_m the maximiser and d = 2T / (g + sqrt(g^2 + 4 b T)),
 * g = |d(ax - bx^2)/dx| at x_m: the distance at which the concave exponent has dropped by T. */
double orc_ln_dist_marg(double d_ref, double d_min, double d_max, double a, double b)
{
    const double T = 80.0;
    const int NP = 200;
    const double xlo = d_ref / d_max, xhi = d_ref / d_min;
    const double lnC = log(3.0 * d_ref * d_ref * d_ref / (d_max * d_max * d_max - d_min * d_min * d_min));
    double xm;
    if (b > 0.0)
        xm = a / (2.0 * b);
    else
        xm = a > 0.0 ? xhi : xlo;
    if (xm < xlo)
        xm = xlo;
    if (xm > xhi)
        xm = xhi;
    const double phim = a * xm - b * xm * xm;
    const double g = fabs(a - 2.0 * b * xm);
    const double den = g + sqrt(g * g + 4.0 * b * T);
    double L = xlo, R = xhi;
    if (den > 0.0) {
        const double d = 2.0 * T / den;
        if (xm - d > L)
            L = xm - d;
        if (xm + d < R)
            R = xm + d;
    }
    const double ul = log(L), h = (log(R) - ul) / NP;
    double s = 0.0;
    for (int p = 0; p < NP; ++p) {
        const double c0 = ul + (p + 0.5) * h;
        for (int i = 0; i < 16; ++i) {
            const double u = c0 + 0.5 * h * orc_gl_t[i];
            const double x = exp(u);
            s += 0.5 * h * orc_gl_w[i] * exp(a * x - b * x * x - 3.0 * u - phim);
        }
    }
    return lnC + phim + log(s);
}

int orc_lnL_one(const orc_problem *P, const double *theta_in, double *lnL_t, double *lnL_tmarg, double *quad_out)
{
    int K = P->n_det, M = P->n_modes;
    double complex F[8], Ylm[64], c[8 * 64];
    double dt[8];
    double theta[6];
    memcpy(theta, theta_in, sizeof(theta));
    if (P->dist_marg)
        theta[5] = P->d_ref;   /* coefficients at x = 1: lin and quad are a and b */
    orc_coeffs(P, theta, F, Ylm, c, dt);
    double quad = orc_quad(P, c);
    double *vals = malloc(sizeof(double) * (size_t)P->n_t);
    if (!vals)
        return -2;
    double mx = -INFINITY;
    for (int j = 0; j < P->n_t; ++j) {
        double lin;
        if (orc_data_term(P, c, dt, j, &lin) != 0) {
            free(vals);
            return -1;
        }
        vals[j] = P->dist_marg ? orc_ln_dist_marg(P->d_ref, P->d_min, P->d_max, lin, quad) : lin - quad;
        if (vals[j] > mx)
            mx = vals[j];
    }
    double s = 0.0;
    for (int j = 0; j < P->n_t; ++j)
        s += exp(vals[j] - mx);
    if (lnL_t)
        memcpy(lnL_t, vals, sizeof(double) * (size_t)P->n_t);
    *lnL_tmarg = mx + log(s) - log((double)P->n_t);
    if (quad_out)
        *quad_out = quad;
    (void)K;
    (void)M;
    free(vals);
    return 0;
}

/* Batch over samples: theta [n][6]; lnL_t [n][n_t] or NULL; quad [n] or NULL.
 * Returns the number of samples whose Q window was exceeded (their outputs are NaN). */
int64_t orc_lnL_batch(const orc_problem *P, const double *theta, int64_t n, double *lnL_t,
                      double *lnL_tmarg, double *quad)
{
    if (P->n_det > 8 || P->n_modes > 64)
        return -1;
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (int64_t i = 0; i < n; ++i) {
        double q;
        int rc = orc_lnL_one(P, theta + 6 * i, lnL_t ? lnL_t + i * P->n_t : NULL, lnL_tmarg + i, &q);
        if (rc != 0) {
            lnL_tmarg[i] = NAN;
            q = NAN;
            ++bad;
        }
        if (quad)
            quad[i] = q;
    }
    return bad;
}

/* Per-sample coefficients for inspection: F [n][K], Y [n][M], c [n][K][M]
 * (complex128 interleaved), dt [n][K]. */
void orc_coeffs_batch(const orc_problem *P, const double *theta, int64_t n, double *F, double *Ylm,
                      double *c, double *dt)
{
    int K = P->n_det, M = P->n_modes;
    for (int64_t i = 0; i < n; ++i) {
        double complex Fi[8], Yi[64], ci[8 * 64];
        orc_coeffs(P, theta + 6 * i, Fi, Yi, ci, dt + i * K);
        for (int k = 0; k < K; ++k) {
            F[2 * (i * K + k)] = creal(Fi[k]);
            F[2 * (i * K + k) + 1] = cimag(Fi[k]);
        }
        for (int m = 0; m < M; ++m) {
            Ylm[2 * (i * M + m)] = creal(Yi[m]);
            Ylm[2 * (i * M + m) + 1] = cimag(Yi[m]);
        }
        for (int q = 0; q < K * M; ++q) {
            c[2 * (i * K * M + q)] = creal(ci[q]);
            c[2 * (i * K * M + q) + 1] = cimag(ci[q]);
        }
    }
}

/* ---------------------------------------------------------------- Monte Carlo reduction */

/* Reduction of log-weights ln w_i = ln L_i + ln p_i - ln p_s,i (Eq. (lnL:MonteCarlo)):
 *   out[0] ln Z      = ln( (1/N) sum_i w_i )
 *   out[1] sigma_lnZ = sqrt( sum w^2 / (sum w)^2 - 1/N )   (relative error of the mean)
 *   out[2] n_eff     = sum w / max w                        (Eq. (neff))
 *   out[3] n_ESS     = (sum w)^2 / sum w^2                  (Kish, Sec. IV A)
 *   out[4] max ln w
 * Sums are taken after subtracting max ln w, in sample order. */
void orc_reduce(const double *lnw, int64_t n, double *out)
{
    double mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (lnw[i] > mx)
            mx = lnw[i];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double e = exp(lnw[i] - mx);
        s1 += e;
        s2 += e * e;
    }
    double var = s2 / (s1 * s1) - 1.0 / (double)n;
    out[0] = mx + log(s1) - log((double)n);
    out[1] = sqrt(var > 0.0 ? var : 0.0);
    out[2] = s1;
    out[3] = s1 * s1 / s2;
    out[4] = mx;
}

/* ---------------------------------------------------------------- counter-based RNG */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5): ten rounds of
 * two 32x32->64 multiplies with the key bumped by the Weyl constants
 * between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Uniform double in [0,1) from two 32-bit words: 27 + 26 high bits -> 53-bit mantissa. */
static double orc_u53(uint32_t a, uint32_t b)
{
    uint64_t v = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)v * (1.0 / 9007199254740992.0);
}

/* The six uniforms of sample i in batch `iter`:
 * counter = (i low word, i high word, iter, p) for p = 0,1,2, key = (seed low, seed high);
 * words (0,1) give dimension 2p, words (2,3) dimension 2p+1. */
void orc_uniforms(uint64_t seed, uint32_t iter, int64_t i, double u[6])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t p = 0; p < 3; ++p) {
        uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, p};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        u[2 * p] = orc_u53(r[0], r[1]);
        u[2 * p + 1] = orc_u53(r[2], r[3]);
    }
}

/* ---------------------------------------------------------------- adaptive Cartesian sampler */

/* Product-form sampling prior (Sec. II B).  Each of the six extrinsic
 * coordinates is sampled through v_d in [0,1), the prior's CDF coordinate,
 * so that the prior is uniform on the unit cube:
 *   alpha = 2 pi v, sin(delta) = 2v - 1, psi = pi v, phi = 2 pi v,
 *   cos(iota) = 1 - 2v, D^3 = D_min^3 + v (D_max^3 - D_min^3).
 * p_s,d is piecewise constant on B equal bins of v_d with masses P[d][b];
 * p(theta)/p_s(theta) = prod_d 1/(B P[d][b_d] / sum_b P[d][b]).
 * Drawing: the bin is the last b with C[b] <= u * C[B] (C the running sum of
 * P, C[0] = 0), and v = (b + (u C[B] - C[b]) / P[b]) / B, the within-bin
 * fraction clamped to [0, 1). */
void orc_draw(const double *P, int B, uint64_t seed, uint32_t iter, int64_t i0, int64_t n,
              double d_min, double d_max, int marg, double *theta, double *lnp_minus_lnps, int32_t *bins,
              double *v_out)
{
    double *C = malloc(sizeof(double) * 6 * (size_t)(B + 1));
    for (int d = 0; d < 6; ++d) {
        C[d * (B + 1)] = 0.0;
        for (int b = 0; b < B; ++b)
            C[d * (B + 1) + b + 1] = C[d * (B + 1) + b] + P[d * B + b];
    }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        double u[6], v[6];
        orc_uniforms(seed, iter, i0 + s, u);
        double lr = 0.0;
        for (int d = 0; d < 6; ++d) {
            const double *Cd = C + d * (B + 1);
            const double *Pd = P + d * B;
            double total = Cd[B];
            double x = u[d] * total;
            int b = 0;
            for (int k = 1; k < B; ++k)
                if (Cd[k] <= x)
                    b = k;
            double t = (x - Cd[b]) / Pd[b];
            if (!(t >= 0.0))
                t = 0.0;
            if (t >= 1.0)
                t = nextafter(1.0, 0.0);
            v[d] = (b + t) / B;
            bins[6 * s + d] = b;
            if (!(marg && d == 5))   /* a marginalised distance carries no sampling weight */
                lr -= log(B * Pd[b] / total);
        }
        double *th = theta + 6 * s;
        th[0] = 2.0 * ORC_PI * v[0];
        th[1] = asin(2.0 * v[1] - 1.0);
        th[2] = ORC_PI * v[2];
        th[3] = 2.0 * ORC_PI * v[3];
        th[4] = acos(1.0 - 2.0 * v[4]);
        th[5] = cbrt(d_min * d_min * d_min + v[5] * (d_max * d_max * d_max - d_min * d_min * d_min));
        lnp_minus_lnps[s] = lr;
        if (v_out)
            for (int d = 0; d < 6; ++d)
                v_out[6 * s + d] = v[d];
    }
    free(C);
}

/* Update of the 1-D marginals after a block of evaluations (Sec. II B):
 *   H[d][b] = sum over samples in bin b of exp(beta (ln w_i - max ln w))
 *   P[d][b] <- (1 - eps) H[d][b] / sum_b H[d][b] + eps / B
 * beta is the tempering exponent, eps the mixing floor.  A dimension whose
 * histogram is empty keeps its previous masses. */
void orc_adapt(double *P, int B, const int32_t *bins, const double *lnw, int64_t n, double eps, double beta,
               int marg)
{
    double mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (lnw[i] > mx)
            mx = lnw[i];
    double *H = calloc(6 * (size_t)B, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        double w = exp(beta * (lnw[i] - mx));
        for (int d = 0; d < 6; ++d)
            H[d * B + bins[6 * i + d]] += w;
    }
    for (int d = 0; d < (marg ? 5 : 6); ++d) {   /* a marginalised distance keeps its masses */
        double tot = 0.0;
        for (int b = 0; b < B; ++b)
            tot += H[d * B + b];
        if (!(tot > 0.0) || !isfinite(tot))
            continue;
        for (int b = 0; b < B; ++b)
            P[d * B + b] = (1.0 - eps) * H[d * B + b] / tot + eps / B;
    }
    free(H);
}

/* ---------------------------------------------------------------- adaptive-volume draws */

/* Draws of the adaptive-volume integrator (Sec. IV A): uniform over the union of the
 * active cells of a grid with 2^level cells per side of the unit cube of prior-CDF
 * coordinates.  A cell's key packs its six integer coordinates, coordinate d in bits
 * [level d, level (d+1)); cells[] holds the active keys in increasing order.
 * Random words of draw i in iteration `iter`: Philox4x32-10 with key = seed and counter
 * (i low, i high, iter, p), p = 0..3; p = 0 words (0,1) give the 53-bit integer U of the
 * cell choice, the cell being cells[floor(U n_cells / 2^53)]; the remaining word pairs in
 * order give the six in-cell uniforms.  v_d = (coordinate_d + u_d) / 2^level, and theta
 * follows from v as for the histogram sampler. */
void orc_av_draw(const uint64_t *cells, int64_t n_cells, int level, uint64_t seed, uint32_t iter, int64_t i0,
                 int64_t n, double d_min, double d_max, double *theta, double *v_out)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double side = ldexp(1.0, level);
    const uint64_t mask = level > 0 ? ((uint64_t)1 << level) - 1 : 0;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        const int64_t i = i0 + s;
        uint32_t w[16];
        for (uint32_t p = 0; p < 4; ++p) {
            const uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, p};
            orc_philox4x32_10(ctr, key, w + 4 * p);
        }
        const uint64_t U = ((uint64_t)(w[0] >> 5) << 26) | (uint64_t)(w[1] >> 6);
        const int64_t c = (int64_t)(((unsigned __int128)U * (uint64_t)n_cells) >> 53);
        const uint64_t cell = cells[c];
        double *v = v_out + 6 * s;
        for (int d = 0; d < 6; ++d) {
            const double u = orc_u53(w[2 + 2 * d], w[3 + 2 * d]);
            const double coord = (double)((cell >> (level * d)) & mask);
            v[d] = (coord + u) / side;
        }
        double *th = theta + 6 * s;
        th[0] = 2.0 * ORC_PI * v[0];
        th[1] = asin(2.0 * v[1] - 1.0);
        th[2] = ORC_PI * v[2];
        th[3] = 2.0 * ORC_PI * v[3];
        th[4] = acos(1.0 - 2.0 * v[4]);
        th[5] = cbrt(d_min * d_min * d_min + v[5] * (d_max * d_max * d_max - d_min * d_min * d_min));
    }
}

/* ---------------------------------------------------------------- portfolio member choice */

/* The portfolio integrator (Sec. IV, "Portfolio integrator") draws each sample from one
 * member, with the members' weights normalised to sum 1.  Draw i of portfolio iteration
 * `iter` uses Philox4x32-10 with key = seed and counter (i low, i high, iter, 7): words
 * (0,1) give the 53-bit integer U, and with x = U 2^-53 the sample comes from member 0
 * when x < t0, from member 1 when t0 <= x < t1, else from member 2 (t0 = W0, t1 = W0 + W1,
 * or a value above 1 when member 2 is not active; exact comparisons in double precision). */
void orc_portfolio_members(uint64_t seed, uint32_t iter, int64_t n, double t0, double t1, int32_t *member)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, 7u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        const double x = orc_u53(r[0], r[1]);
        member[i] = x < t0 ? 0 : (x < t1 ? 1 : 2);
    }
}

/* ---------------------------------------------------------------- Gaussian-mixture draws */

/* Standard normal CDF and its inverse.  The inverse refines a starting value by Newton's
 * method on Phi (Phi' = the normal density), taking the smaller tail so that the relative
 * precision of p is kept: x with Phi(x) = p to ~1 ulp in a handful of steps. */
static double orc_phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

double orc_ndtri(double p)
{
    if (!(p > 0.0))
        return -INFINITY;
    if (!(p < 1.0))
        return INFINITY;
    const int upper = p > 0.5;
    const double q = upper ? 1.0 - p : p;   /* exact for p > 0.5 */
    /* x < 0 with Phi(x) = q: start from the tail asymptote, then Newton on Phi */
    double x = -sqrt(-2.0 * log(q));   /* the tail asymptote (below the root) */
    for (int it = 0; it < 100; ++it) {
        const double f = orc_phi(x) - q;
        const double d = exp(-0.5 * x * x) / sqrt(2.0 * ORC_PI);
        if (!(d > 0.0))
            break;
        const double step = f / d;
        x -= step;
        if (fabs(step) <= 1e-16 * fmax(1.0, fabs(x)))
            break;
    }
    return upper ? -x : x;
}

/* Draws of the Gaussian-mixture sampling prior on the unit cube of prior-CDF coordinates:
 * C components with weights pi[c], per-dimension means mu[c][d] in [0, 1] and widths
 * sig[c][d] (diagonal covariances), each dimension truncated to [0, 1].  Draw i of
 * iteration `iter`: Philox4x32-10 with key = seed and counter (i low, i high, iter, p);
 * p = 8: words (0,1) give the 53-bit U of the component, the first c with
 * U 2^-53 < pi[0] + ... + pi[c] (pi normalised to sum 1, the last component otherwise);
 * p = 9, 10, 11: word pairs (0,1), (2,3) give the six uniforms u_d, and
 * v_d = mu + sig Phi^-1(Phi(a) + u_d (Phi(b) - Phi(a))), a = -mu/sig, b = (1 - mu)/sig,
 * kept in [0, 1).  theta follows from v as for the histogram sampler. */
void orc_gmm_draw(const double *pi, const double *mu, const double *sig, int C, uint64_t seed, uint32_t iter,
                  int64_t n, double d_min, double d_max, double *theta, double *v_out, int32_t *comp)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double tot = 0.0;
    for (int c = 0; c < C; ++c)
        tot += pi[c];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t r[4];
        uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, 8u};
        orc_philox4x32_10(ctr, key, r);
        const double U = orc_u53(r[0], r[1]);
        int c = C - 1;
        double run = 0.0;
        for (int k = 0; k < C - 1; ++k) {
            run += pi[k] / tot;
            if (U < run) {
                c = k;
                break;
            }
        }
        double u[6], v[6];
        for (uint32_t p = 0; p < 3; ++p) {
            ctr[3] = 9u + p;
            orc_philox4x32_10(ctr, key, r);
            u[2 * p] = orc_u53(r[0], r[1]);
            u[2 * p + 1] = orc_u53(r[2], r[3]);
        }
        for (int d = 0; d < 6; ++d) {
            const double m = mu[c * 6 + d], s = sig[c * 6 + d];
            const double pa = orc_phi(-m / s), pb = orc_phi((1.0 - m) / s);
            double x = m + s * orc_ndtri(pa + u[d] * (pb - pa));
            if (!(x >= 0.0))
                x = 0.0;
            if (x >= 1.0)
                x = nextafter(1.0, 0.0);
            v[d] = x;
        }
        double *th = theta + 6 * i;
        th[0] = 2.0 * ORC_PI * v[0];
        th[1] = asin(2.0 * v[1] - 1.0);
        th[2] = ORC_PI * v[2];
        th[3] = 2.0 * ORC_PI * v[3];
        th[4] = acos(1.0 - 2.0 * v[4]);
        th[5] = cbrt(d_min * d_min * d_min + v[5] * (d_max * d_max * d_max - d_min * d_min * d_min));
        for (int d = 0; d < 6; ++d)
            v_out[6 * i + d] = v[d];
        comp[i] = c;
    }
}

/* ---------------------------------------------------------------- fair draws */

/* The final ILE pass (Sec. II, the closing paragraph of the method overview, and the
 * two-step posterior construction of Sec. II D): extrinsic samples are drawn fairly,
 * with replacement, from the Monte Carlo integral's weighted samples, and each draw's
 * time from the per-bin likelihood of that sample (the time prior is uniform on the grid).
 *
 * Readings where the paper is silent:
 *  - every discrete choice is made exactly in integer arithmetic.  Item i of a list of
 *    log-weights x gets W_i = floor(exp(x_i - max x) 2^S) with S = 62 - ceil(log2 n)
 *    (0 for non-finite x_i), so the total stays below 2^62;
 *  - draw d uses Philox4x32-10 with key = seed and counter = (d low, d high,
 *    0xFFFFFFFF, 0); words (0,1) give the 53-bit integer U of the sample choice, words
 *    (2,3) that of the time choice (the same 27 + 26 bit split as orc_u53);
 *  - the chosen item is the first whose running sum of W exceeds floor(U Total / 2^53). */
static int orc_fix_shift(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n)
        ++c;
    return 62 - c;
}

static uint64_t orc_fix_weight(double x, double mx, int S)
{
    if (!isfinite(x))
        return 0;
    return (uint64_t)ldexp(exp(x - mx), S);
}

/* 53-bit integers (sample choice, time choice) of draw d. */
void orc_fair_words(uint64_t seed, int64_t d, uint64_t U[2])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(uint64_t)d, (uint32_t)((uint64_t)d >> 32), 0xFFFFFFFFu, 0u};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    U[0] = ((uint64_t)(r[0] >> 5) << 26) | (uint64_t)(r[1] >> 6);
    U[1] = ((uint64_t)(r[2] >> 5) << 26) | (uint64_t)(r[3] >> 6);
}

/* Running sums of the fixed-point weights of x[0..n); returns the shift S, or -1 if no
 * x is finite.  cum has n entries. */
int orc_fix_cumulative(const double *x, int64_t n, uint64_t *cum)
{
    double mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (isfinite(x[i]) && x[i] > mx)
            mx = x[i];
    if (!isfinite(mx))
        return -1;
    const int S = orc_fix_shift(n);
    uint64_t run = 0;
    for (int64_t i = 0; i < n; ++i) {
        run += orc_fix_weight(x[i], mx, S);
        cum[i] = run;
    }
    return S;
}

/* First i with cum[i] > floor(U cum[n-1] / 2^53) (binary search over the running sums). */
int64_t orc_fix_choose(const uint64_t *cum, int64_t n, uint64_t U)
{
    const uint64_t T = (uint64_t)(((unsigned __int128)U * cum[n - 1]) >> 53);
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (cum[mid] > T)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* n_draws fair draws from the weighted samples lnw[0..n): sample indices idx[] and the
 * time-choice integers U_time[] (for the second step).  Returns 0, or -1 if no weight is
 * finite. */
int orc_fair_draws(const double *lnw, int64_t n, uint64_t seed, int64_t n_draws, int64_t *idx, uint64_t *U_time)
{
    uint64_t *cum = malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (n < 1 || orc_fix_cumulative(lnw, n, cum) < 0) {
        free(cum);
        return -1;
    }
    for (int64_t d = 0; d < n_draws; ++d) {
        uint64_t U[2];
        orc_fair_words(seed, d, U);
        idx[d] = orc_fix_choose(cum, n, U[0]);
        U_time[d] = U[1];
    }
    free(cum);
    return 0;
}

/* Time bin of one draw from its per-bin ln L[0..n_t) and its time-choice integer. */
int64_t orc_fair_time_bin(const double *lnL_bins, int64_t n_t, uint64_t U)
{
    uint64_t *cum = malloc(sizeof(uint64_t) * (size_t)n_t);
    int64_t j = -1;
    if (orc_fix_cumulative(lnL_bins, n_t, cum) >= 0)
        j = orc_fix_choose(cum, n_t, U);
    free(cum);
    return j;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
