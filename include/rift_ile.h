/*
 * rift_ile.h - C ABI of the GB300 (sm_103a) library for the extrinsic-marginalised
 * likelihood integral (ILE) of arXiv:2505.11655 ("Narrowing RIFT").
 *
 * For one intrinsic point the library takes the per-detector mode overlaps
 * Q_k,lm(t) and the Gram matrices U_k, V_k (Sec. II A, Eq. (QUV)) and, for
 * extrinsic samples theta = (alpha, delta, psi, phi, iota, D), evaluates
 *
 *   ln L(theta, t) = (D_ref/D) Re sum_k sum_lm conj(F_k Y_lm) Q_k,lm(t + dt_k)
 *                    - kappa (D_ref/D)^2 sum_k sum_lm,l'm' [ |F_k|^2 conj(Y_lm) Y_l'm' U_k
 *                                                           + Re(F_k^2 Y_lm Y_l'm' V_k) ]
 *   (Sec. II A, Eq. (def:lnL:Decomposed); kappa = 1/4 as printed),
 *
 * marginalises it over a uniform grid of geocentric times (App. timing: every
 * evaluation is time marginalised), and reduces exp(ln L) p/p_s over samples
 * to ln Z, n_eff and n_ESS (Sec. II B Eq. (lnL:MonteCarlo); Sec. II C
 * Eq. (neff); Sec. IV A).  Samples come from a product-form adaptive
 * histogram sampling prior kept on the device (Sec. II B, "adaptive
 * Cartesian" integrator).
 *
 * Conventions (all entry points):
 *   - Every function returns an int status: RIFT_OK (0) or a negative RIFT_E* code.
 *     No C++ exception crosses this boundary.  rift_ile_strerror() names a code.
 *   - A handle is used by one host thread at a time.  Its work is ordered on the
 *     CUDA stream given at creation (NULL = the legacy default stream).
 *   - Pointers tagged with a `mem` argument are host memory (RIFT_MEM_HOST) or
 *     device memory of the handle's GPU (RIFT_MEM_DEVICE).  The caller owns them
 *     and keeps them valid until the call returns; calls with device outputs
 *     return after the results are written (they synchronise the stream).
 *   - Complex arrays are interleaved (re, im) float64 pairs ("complex128").
 *   - The handle owns every device buffer it allocates; rift_ile_destroy frees them.
 */
#ifndef RIFT_ILE_H
#define RIFT_ILE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define RIFT_OK 0
#define RIFT_EINVAL -1     /* invalid argument, size or configuration                          */
#define RIFT_ENOMEM -2     /* device or host allocation failed                                  */
#define RIFT_ECUDA -3      /* a CUDA runtime call or kernel launch failed                       */
#define RIFT_ERANGE -4     /* a time-shifted Q interpolation node would leave the Q window      */
#define RIFT_ENONFINITE -5 /* a NaN or infinity reached the likelihood or its reduction        */
#define RIFT_ETIMEOUT -6   /* a bounded device wait gave up                                     */
#define RIFT_ESTATE -7     /* call out of order (e.g. no overlaps set) or a bad state blob      */

/* ---- enumerations ---------------------------------------------------------------------- */
#define RIFT_MEM_HOST 0
#define RIFT_MEM_DEVICE 1

#define RIFT_QUAD_QUARTER 0 /* kappa = 1/4, as printed in Eq. (def:lnL:Decomposed) */
#define RIFT_QUAD_HALF 1    /* kappa = 1/2 (equivalent to QUARTER with U, V doubled)  */

#define RIFT_FP64 0  /* every step in float64: the plain reference GPU path               */
#define RIFT_FP32 1  /* float32 bulk arithmetic; float64 delays, log-sum-exp and sums; the  */
                     /* samples with large data and template terms corrected in           */
                     /* double-float, so every ln L is within 1e-3 of the float64 value   */
                     /* at moderate SNR (measured: 5e-4 at SNR 20; at SNR 150 the other   */
                     /* bins' data terms of ~1e4 keep their float32 rounding, ~1.3e-3)    */
#define RIFT_MIXED 2 /* FP32, then float64 re-evaluation of the samples that carry weight  */
                     /* (ln w within 40 of the batch's largest): those to the float64     */
                     /* path's accuracy, the others as RIFT_FP32                          */

#define RIFT_MAX_DET 4
#define RIFT_MAX_MODES 32
#define RIFT_MAX_ITER 64
#define RIFT_MAX_BINS 1024

typedef struct rift_ile rift_ile_t;

/* Problem description.  All pointers are HOST memory, copied during
 * rift_ile_create; the caller keeps ownership.
 *
 *   det_tensor [n_det][3][3]  detector response tensors D_k (Earth-fixed frame)
 *   det_pos_m  [n_det][3]     detector vertex positions x_k (m); dt_k = -x_k . n / c (Sec. II A)
 *   gmst_rad                  Greenwich sidereal angle of the reference epoch (an input)
 *   lm         [n_modes][2]   (l, m) of each mode; 2 <= l <= 6, |m| <= l, no duplicates
 *   fs_hz, n_q, q_t0_s[n_det] Q_k,lm is sampled at q_t0_s[k] + i / fs_hz, i = 0..n_q-1
 *                             (seconds relative to the reference epoch)
 *   t_lo_s, t_hi_s, n_t       geocentric time grid t_j = t_lo + j (t_hi - t_lo)/(n_t - 1),
 *                             the time marginal is the mean of exp(ln L) over it
 *   d_ref_mpc                 D_ref of Eq. (strain_mode); d_min/max the distance prior range
 *   quad_norm                 RIFT_QUAD_QUARTER or RIFT_QUAD_HALF
 *   precision                 RIFT_FP64, RIFT_FP32 or RIFT_MIXED
 *   n_bins                    histogram bins per dimension of the sampling prior (2..1024)
 *   adapt_floor               mixing floor eps in [0, 1): P <- (1-eps) H/sum H + eps/B
 *   adapt_temper              exponent beta > 0 applied to the weights when adapting
 *   seed                      key of the counter-based generator (Philox4x32-10)
 *   max_samples               largest sample batch of one iteration (sizes device buffers)
 *   distance_marg             0: the distance is sampled.  1: it is marginalised in every
 *                             time bin: ln L is exactly a x - b x^2 in x = D_ref/D (a, b the
 *                             data and template terms at D = D_ref), and each bin's value is
 *                             ln int p(D) e^{a x - b x^2} dD with p(D) = 3 D^2/(D_max^3 - D_min^3)
 *                             on [d_min, d_max], by Gauss-Legendre quadrature in ln x over the
 *                             range where the exponent is within 18 (float32: 2 panels of 10
 *                             nodes) or 44 (float64: 4 panels of 16) of its maximum; the
 *                             sampler's distance coordinate then carries no weight and keeps
 *                             its masses (theta[5] of the draws is not used).  The paper only
 *                             mentions distance marginalisation; this quadrature is this
 *                             library's.  rift_ile_av and rift_ile_fair_draws refuse it.
 *
 * Validation: RIFT_EINVAL for bad sizes or modes; RIFT_ERANGE unless, for every
 * detector and every sky position, t_lo - |x_k|/c and t_hi + |x_k|/c map inside
 * [q_t0_s[k], q_t0_s[k] + (n_q - 2)/fs_hz] (a Q index outside the window is an error,
 * never a clamp). */
typedef struct {
    int32_t n_det;
    const double *det_tensor;
    const double *det_pos_m;
    double gmst_rad;
    int32_t n_modes;
    const int32_t *lm;
    double fs_hz;
    int32_t n_q;
    const double *q_t0_s;
    double t_lo_s, t_hi_s;
    int32_t n_t;
    double d_ref_mpc, d_min_mpc, d_max_mpc;
    int32_t quad_norm;
    int32_t precision;
    int32_t n_bins;
    double adapt_floor;
    double adapt_temper;
    uint64_t seed;
    int64_t max_samples;
    int32_t distance_marg;
} rift_ile_config;

/* Result of a marginalisation or an adaptive run (host struct, filled by the call).
 * Pooled values use every sample of every iteration of the call, each weighted
 * by the sampling prior it was drawn from:
 *   lnZ = ln( (1/N) sum_i w_i ),  w_i = L_tmarg,i p_i / p_s,i      (Eq. (lnL:MonteCarlo))
 *   sigma_lnZ = sqrt( sum w^2 / (sum w)^2 - 1/N )                   (relative error of the mean)
 *   n_eff = sum w / max w                                           (Eq. (neff))
 *   n_ess = (sum w)^2 / sum w^2                                     (Sec. IV A)
 *   lnL_max = largest time-marginalised ln L seen.
 * *_iter[g] are the same quantities for iteration g alone.  time_ms[]: device
 * time of the call measured with CUDA events (0 draw+sort, 1 likelihood,
 * 2 reduce+adapt, 3 whole call). */
typedef struct {
    double lnZ, sigma_lnZ, n_eff, n_ess, lnL_max;
    int64_t n_total;
    int32_t n_iter;
    int32_t status;
    double lnZ_iter[RIFT_MAX_ITER];
    double sigma_iter[RIFT_MAX_ITER];
    double n_eff_iter[RIFT_MAX_ITER];
    double n_ess_iter[RIFT_MAX_ITER];
    double time_ms[4];
} rift_ile_result;

/* Create a handle: validate `cfg`, copy it, allocate device buffers for
 * cfg->max_samples samples.  `cuda_stream` is a cudaStream_t (or NULL).
 * On error *out is NULL and nothing stays allocated. */
int rift_ile_create(const rift_ile_config *cfg, void *cuda_stream, rift_ile_t **out);

/* Set Q [n_det][n_modes][n_q], U and V [n_det][n_modes][n_modes] (complex128,
 * Sec. II A Eq. (QUV)).  The library keeps float64 copies and a float32
 * split-plane copy of Q (plane 2m = Re Q_m, plane 2m+1 = Im Q_m).
 * RIFT_EINVAL unless U_k is Hermitian and V_k symmetric to 1e-10 relative to
 * their largest entry (Sec. V A symmetry relations); RIFT_ENONFINITE on NaN/Inf. */
int rift_ile_set_overlaps(rift_ile_t *h, const void *Q, const void *U, const void *V, int mem);

/* Overlaps from frequency-domain inputs, computed on the device (Sec. II A, Eq. QUV; the
 * precompute stage the paper runs on the CPU): on a two-sided grid of n_freq frequencies
 * f_j, mirror symmetric (f[n_freq-1-j] == -f[j] exactly), with inverse-PSD weights
 * w_k(f) symmetric in f,
 *   Q_k,lm(t_s)  = 2 sum_j w_k(f_j) exp(2 pi i f_j t_s) conj(h_lm(f_j)) d_k(f_j),
 *                  t_s = q_t0_s[k] + s / fs_hz, s = 0 .. n_q - 1,
 *   U_k,lm,l'm'  = 2 sum_j w_k conj(h_lm) h_l'm',  V_k,lm,l'm' = 2 sum_j w_k h_lm(-f_j) h_l'm'(f_j)
 * (only lm <= l'm' is summed; U is mirrored Hermitian, V symmetric), then installed as
 * rift_ile_set_overlaps would install them.  All in float64.
 *   freqs [n_freq] (Hz), hlm [n_modes][n_freq] complex128 (mode waveforms shared by the
 *   detectors), data [n_det][n_freq] complex128, weights [n_det][n_freq]; all in `mem`,
 *   read during the call (scratch about 16 n_det n_modes n_freq bytes from the pool).
 * RIFT_EINVAL for a grid that is not mirror symmetric or weights that are negative or not
 * symmetric; RIFT_ENONFINITE for non-finite weights or overlaps. */
int rift_ile_set_waveforms(rift_ile_t *h, int32_t n_freq, const double *freqs, const void *hlm, const void *data,
                           const double *weights, int mem);

/* Copy the installed float64 overlaps out: Q [n_det][n_modes][n_q], U, V [n_det][n_modes]
 * [n_modes] complex128 in `mem` (any may be NULL).  RIFT_ESTATE before overlaps are set. */
int rift_ile_get_overlaps(const rift_ile_t *h, void *Q, void *U, void *V, int mem);

/* Evaluate n samples theta [n][6] = (alpha, delta, psi, phi, iota, D):
 *   lnL_tmarg [n]      time-marginalised ln L = ln( (1/n_t) sum_j exp(ln L(theta, t_j)) )
 *   lnL_t [n][n_t]     ln L at every bin, or NULL
 * theta and the outputs live in `mem`.  Any n >= 0 is accepted (processed in
 * batches of max_samples).  Uses the handle's precision mode. */
int rift_ile_eval(rift_ile_t *h, const double *theta, int64_t n, int mem, double *lnL_tmarg, double *lnL_t);

/* Per-sample ingredients of the likelihood for inspection and parity checks:
 *   c [n][n_det][n_modes] complex128 = (D_ref/D) F_k Y_lm(iota, -phi),
 *   dt [n][n_det] arrival delays (s), quad [n] the template (quadratic) term.
 * Any output may be NULL.  Computed in float64 in RIFT_FP64 mode, float32 otherwise. */
int rift_ile_coeffs(rift_ile_t *h, const double *theta, int64_t n, int mem, double *c, double *dt, double *quad);

/* One Monte Carlo batch: draw n_samples from the current sampling prior (no
 * adaptation), evaluate, reduce.  1 <= n_samples <= max_samples. */
int rift_ile_marginalize(rift_ile_t *h, int64_t n_samples, rift_ile_result *out);

/* n_iter iterations of draw -> evaluate -> reduce -> adapt, all on the device;
 * results pooled over the iterations (see rift_ile_result). 1 <= n_iter <= RIFT_MAX_ITER.
 * When a call repeats the previous call's (n_iter, n_per_iter), the whole sequence is
 * captured once as a CUDA graph and replayed by later calls of that shape (same
 * kernels and arguments; the sampler's iteration counter lives in device memory).
 * RIFT_ILE_GRAPHS=0 in the environment turns the capture off. */
int rift_ile_adapt(rift_ile_t *h, int32_t n_iter, int64_t n_per_iter, rift_ile_result *out);

/* Launch plan of the float32 likelihood stage for the most recent batch:
 * *lnl_kernel = RIFT_KERNEL_FP64 (RIFT_FP64 mode), RIFT_KERNEL_CUDA_CORE (64-sample
 * CUDA-core tiles) or RIFT_KERNEL_TENSOR (128-sample tcgen05 tiles);
 * *samples_per_cell = fill of the Hilbert sky-sort grid.  The plan is picked per
 * problem class by the autotuner (timed candidates on the first batch of a class;
 * RIFT_ILE_TUNE=0 disables the timing, RIFT_ILE_TUNE_CACHE=<file> persists the
 * choices) unless RIFT_ILE_TC=0/1 forces the kernel; RIFT_ILE_DELAY3=0/1 forces the sort key
 * of problems with three or more detectors (sky curve, or Morton key of three delays).  Either output may be NULL. */
#define RIFT_KERNEL_FP64 0
#define RIFT_KERNEL_CUDA_CORE 1
#define RIFT_KERNEL_TENSOR 2
int rift_ile_get_plan(const rift_ile_t *h, int32_t *lnl_kernel, int32_t *samples_per_cell);

/* Samples of the most recent batch (in draw order): theta [n][6], ln p - ln p_s [n],
 * time-marginalised ln L [n], ln w [n]; any output may be NULL; *n_out receives
 * the batch size.  For parity checks of the device's own sample stream. */
int rift_ile_last_batch(rift_ile_t *h, int mem, double *theta, double *lnp_minus_lnps, double *lnL_tmarg,
                        double *lnw, int64_t *n_out);

/* Adaptive-volume integrator (arXiv:2505.11655 Sec. IV A, the paper's recommended ILE
 * integrator), an alternative to rift_ile_adapt's histogram sampler.  It works on the unit
 * cube of prior-CDF coordinates (the same coordinates the histogram sampler draws through)
 * with nested grids of 2^level cells per side (level <= 10):
 *   1. n_per_iter draws uniform over the active cells (ln p - ln p_s = ln V, V their volume);
 *   2. time-marginalised ln L in the handle's precision;
 *   3. the draws passing the current threshold join the live set (draw order, at most
 *      `capacity` live points);
 *   4. the threshold keeps the fewest top 1/64-wide ln L bins (below the live maximum)
 *      holding both the fraction p_thr of the live mass and at least n_min_star points
 *      (n_min_star is a floor: while a few points carry p_thr of the mass, the top
 *      n_min_star set the threshold); masses are exact fixed-point integers;
 *   5. refinement: with V_thr the estimated volume above the current threshold (1 at the
 *      start), V' = V_thr N_min / N_live, dV = V' / sqrt(N_min), n_bins = (1/dV)^(1/6)
 *      (Eq. nbins_V) rounded down to a power of two and never coarser, V_thr <- V'; the
 *      new active cells are the cells holding a kept live point.
 * Draw i of AV iteration g uses Philox4x32-10 with key = seed and counter
 * (i low, i high, g, p), p = 0..3: the first word pair chooses the cell (first of the
 * sorted active cells at floor(U n_cells / 2^53)), the next six the in-cell uniforms.
 * Results pool every iteration's draws (ln w = ln L + ln V) like rift_ile_adapt; the last
 * iteration's draws are the handle's most recent batch (rift_ile_last_batch,
 * rift_ile_fair_draws).  restart = 1 (or the first call) starts from the whole cube; the
 * live set's device memory (about 130 B per point of `capacity`) is allocated by the
 * first call and `capacity` cannot change afterwards (RIFT_EINVAL).
 * RIFT_EINVAL for n_iter outside 1..RIFT_MAX_ITER, n_per_iter outside 1..max_samples,
 * p_thr outside (0, 1], n_min_star < 1, capacity < n_per_iter or >= 2^31 - 2. */
int rift_ile_av(rift_ile_t *h, int32_t n_iter, int64_t n_per_iter, double p_thr, int64_t n_min_star,
                int64_t capacity, int32_t restart, rift_ile_result *out);
/* State of the adaptive-volume integrator after the last call: grid level, active cells,
 * live points, active volume.  Any output may be NULL. */
int rift_ile_av_info(const rift_ile_t *h, int32_t *level, int64_t *n_cells, int64_t *n_live, double *volume);

/* Portfolio integrator (arXiv:2505.11655 Sec. IV, "Portfolio integrator"): the sampling
 * prior is the weighted average of its members' priors, p_s = sum_a W_a p_s,a with
 * sum_a W_a = 1 over the active members, here over the histogram sampler (member 0:
 * rift_ile_adapt's, the handle's masses), the adaptive-volume integrator (member 1:
 * rift_ile_av's, the handle's AV state) and a Gaussian-mixture sampling prior (member 2:
 * the GMM sampler Sec. II B names; its state is held by the handle).  All draw through the
 * prior-CDF cube, where their densities relative to the prior are
 *   g_hist(v) = prod_d B P_d[b_d] / sum_b P_d[b],   g_AV(v) = 1/V on the active cells (0
 *   elsewhere),   g_GMM(v) = sum_c pi_c prod_d phi((v_d - mu_cd)/sig_cd) /
 *   (sig_cd (Phi(b_cd) - Phi(a_cd))),  a = -mu/sig, b = (1 - mu)/sig
 * (C components, diagonal covariances, each dimension truncated to [0, 1]; phi, Phi the
 * standard normal density and CDF).  Portfolio iteration g (counted from the last restart):
 *   1. with x = U 2^-53, U the 53-bit integer of words 0,1 of Philox4x32-10 (key = seed,
 *      counter (i low, i high, g, 7)), draw i comes from member 0 when x < W_0, from member
 *      1 when x < W_0 + W_1, else from member 2 (with one member active, from it); member 0
 *      draws as rift_ile_adapt's iteration g would, member 1 as rift_ile_av's iteration g
 *      would, member 2 with counters (i low, i high, g, 8..11): words 0,1 of counter 8 give
 *      the uniform of the component, the first c whose running sum of pi / sum pi exceeds
 *      it; the word pairs of counters 9..11 the six uniforms u_d, and
 *      v_d = mu_cd + sig_cd Phi^-1(Phi(a_cd) + u_d (Phi(b_cd) - Phi(a_cd))) (kept in [0, 1));
 *   2. ln p - ln p_s = -ln(sum over the active members of W_a g_a(v)) (the bin of another
 *      member's draw is floor(v_d B)); with one member active, that member's own value;
 *   3. time-marginalised ln L, ln w, the iteration's record;
 *   4. weights (adapt_weights = 1, two or more members active): n_ESS,a = (sum w)^2 /
 *      sum w^2 over the batch's draws from member a; W' proportional to n_ESS; no weight
 *      below 0.05/N_s (N_s the active members): those below are set to it and the others
 *      scaled to fill the rest, until none is below;
 *   5. training: a member whose new weight is below 0.05 is frozen (not trained); member 0
 *      adapts its masses on every sample of the batch (bins, ln w); member 1 updates its
 *      live set, threshold and grid (rift_ile_av steps 3-5) from its own draws in index
 *      order (none: not trained); member 2 takes one weighted EM step on every sample:
 *      omega_i = exp(ln w_i - max ln w), responsibilities r_ic proportional to pi_c g_c(v_i),
 *      S_c = sum_i omega r_ic, S = sum_c S_c; pi_c <- 0.98 S_c / S + 0.02 / C,
 *      mu_cd <- sum omega r v_d / S_c, sig_cd^2 <- sum omega r v_d^2 / S_c - mu_cd^2, mu kept
 *      in [0, 1] and sig in [1e-3, 1]; a component with S_c <= 1e-300 S keeps its mu and
 *      sig; nothing changes when no ln w is finite.
 *   cfg->members        RIFT_MEMBER_HIST | RIFT_MEMBER_AV | RIFT_MEMBER_GMM; at least one
 *                       member active in iteration 0
 *   cfg->av_start       first iteration in which member 1 draws; when it joins at
 *                       av_start > 0 the weights restart from w_init
 *   cfg->gmm_start      the same for member 2
 *   cfg->gmm_components C of member 2, 1..RIFT_GMM_MAX_COMPONENTS; its initial state is
 *                       pi_c = 1/C, sig = 0.25, mu_cd = frac((c + 1/2) frac(sqrt(p_d))) with
 *                       p_d = 2, 3, 5, 7, 11, 13
 *   cfg->adapt_weights  1: step 4; 0: the weights stay at w_init
 *   cfg->w_init[3]      initial weights, finite and > 0 for every member (normalised over
 *                       the active members)
 *   cfg->p_thr, n_min_star, capacity   member 1's settings, as for rift_ile_av (the
 *                       capacity is fixed by the first rift_ile_av or portfolio call)
 * restart = 1 (or the first call): weights from w_init, iteration 0, uniform histogram
 * masses, the AV member on the whole cube, the GMM at its initial state; without a restart
 * the members and C must be those of the calls since the last one (else RIFT_EINVAL).
 * Results pool the call's iterations like rift_ile_adapt; the last iteration's draws are
 * the handle's most recent batch.  Not with distance_marg.  RIFT_EINVAL for bad arguments
 * (as rift_ile_av, and the above). */
#define RIFT_MEMBER_HIST 1
#define RIFT_MEMBER_AV 2
#define RIFT_MEMBER_GMM 4
#define RIFT_GMM_MAX_COMPONENTS 16
typedef struct {
    int32_t members;
    int32_t av_start;
    int32_t gmm_start;
    int32_t gmm_components;
    int32_t adapt_weights;
    int32_t reserved;
    double w_init[3];
    double p_thr;
    int64_t n_min_star;
    int64_t capacity;
} rift_portfolio_config;
int rift_ile_portfolio(rift_ile_t *h, int32_t n_iter, int64_t n_per_iter, const rift_portfolio_config *cfg,
                       int32_t restart, rift_ile_result *out);
/* State after the last portfolio iteration: iterations since restart, the weights the
 * last batch was drawn with and those of the next, each member's n_ESS and draw count in
 * the last batch, whether it took part (active) and whether it was frozen (not trained
 * after that batch); entries 0, 1, 2 are members 0, 1, 2. */
typedef struct {
    int32_t iteration;
    int32_t active[3];
    int32_t frozen[3];
    int32_t reserved;
    double W_last[3];
    double W_next[3];
    double n_ess[3];
    int64_t n_drawn[3];
} rift_portfolio_info;
int rift_ile_portfolio_info(const rift_ile_t *h, rift_portfolio_info *info);
/* Member 2's state after the last portfolio iteration (its training included): weights
 * pi [C], means mu [C][6] and widths sig [C][6] in prior-CDF coordinates, host buffers of
 * `capacity` components (outputs may be NULL), C in *n_components (may be NULL).
 * RIFT_ESTATE when no portfolio call since the last restart had the GMM member;
 * RIFT_EINVAL for capacity < C. */
int rift_ile_portfolio_gmm(const rift_ile_t *h, int32_t capacity, int32_t *n_components, double *pi, double *mu,
                           double *sig);

/* Fair draws from the most recent batch (the final ILE pass: extrinsic samples drawn
 * fairly from the Monte Carlo integral's weighted samples, arXiv:2505.11655 Sec. II;
 * the two-step fair draw of Sec. II D).  Draw d takes sample i, with replacement, with
 * probability w_i / sum w (w = exp(ln w) of that batch), then a time bin j with
 * probability exp(ln L(theta_i, t_j)) / sum_j exp(ln L(theta_i, t_j)), the per-bin
 * ln L evaluated in float64 (the time prior is uniform on the grid).
 *   n_draws            number of draws (0 is a no-op)
 *   seed               key of the draws' random numbers (independent of the sampler)
 *   theta [n_draws][6] drawn samples, t [n_draws] their times (s, relative to the
 *                      reference epoch), index [n_draws] their positions in the batch;
 *                      any output may be NULL (not all), all in `mem`.
 * Every choice is exact in integer arithmetic: weights floor(exp(x - max x) 2^S),
 * S = 62 - ceil(log2 count), and the first item whose running sum exceeds
 * floor(U Total / 2^53) for the 53-bit integer U of Philox4x32-10 (key = seed, counter =
 * (d low, d high, 0xFFFFFFFF, 0); words 0,1 for the sample, 2,3 for the time bin).
 * RIFT_ESTATE if there is no batch yet; RIFT_ENONFINITE if a ln w of the batch is not
 * finite; RIFT_ENOMEM if the scratch (about 16 n + 70 n_draws + 16 MiB bytes) cannot be
 * allocated. */
int rift_ile_fair_draws(rift_ile_t *h, int64_t n_draws, uint64_t seed, int mem, double *theta, double *t,
                        int64_t *index);

/* Sampler state (histogram masses, counter, seed) as an opaque versioned blob.
 * get: if buf is NULL, *len receives the size; otherwise *len must be >= it.
 * set: restores a blob from get (RIFT_ESTATE if malformed or of another shape). */
int rift_ile_get_state(const rift_ile_t *h, void *buf, size_t *len);
int rift_ile_set_state(rift_ile_t *h, const void *buf, size_t len);

/* Histogram masses P [6][n_bins] (host) of the current sampling prior. */
int rift_ile_get_sampler(const rift_ile_t *h, double *P);

/* Device bytes a handle created from `cfg` allocates (an upper bound, used for
 * admission control), or -1 if `cfg` is invalid.  Host memory only; no CUDA call. */
int64_t rift_ile_footprint(const rift_ile_config *cfg);

/* Check of the failure path (no counterpart in the paper).  Every wait in the tensor-core
 * kernels is bounded by the GPU's global timer; when a wait runs out the kernel records a
 * timeout in the handle's error word, releases what it holds and returns, and the call
 * reports RIFT_ETIMEOUT with the context still usable.  This call runs that same bounded
 * wait on a barrier that nothing completes, with a limit of limit_ns (1 us .. 2 s), and
 * returns what the host reads back: RIFT_ETIMEOUT when the path works.  RIFT_EINVAL for a
 * limit out of range. */
int rift_ile_wait_selftest(rift_ile_t *h, int64_t limit_ns);

/* Number of kernels this handle has launched since creation (diagnostics: lets a
 * caller count device launches inside a timed region).  Returns -1 for NULL. */
int64_t rift_ile_kernel_launches(const rift_ile_t *h);

/* Reduction of log-weights that allocates nothing (no counterpart in the paper; it
 * exists for callers that cannot allocate device memory at the point of the call:
 * code running under a fixed memory budget or a caching allocator it must not
 * bypass, real-time loops where cudaMalloc's implicit synchronisation is not
 * allowed, or a host that has handed all free device memory to other work).
 *
 *   lnw  [n]  float64 log-weights ln w_i, DEVICE memory (read only)
 *   lnL  [n]  optional float64 values whose maximum is reported in out[5]
 *             (NULL: the maximum of lnw is reported instead)
 *   out  [8]  DEVICE memory, written: ln Z = ln((1/n) sum w), sigma_lnZ, n_eff =
 *             sum w / max w, n_ESS = (sum w)^2 / sum w^2, max ln w, max lnL, n, 0
 *             (the same definitions and kernels as rift_ile_marginalize in RIFT_FP64
 *             mode: every term exp(ln w - max) in float64; the float32 modes of
 *             rift_ile_marginalize sum float32 terms, ~1e-7 relative)
 *   cuda_stream  cudaStream_t (NULL: legacy default stream); the call waits for
 *             the stream before returning, to read its status.
 *
 * Scratch is a 12 KiB file-scope device array inside the library, held by every
 * GPU that loads the library until the process exits; nothing is allocated per
 * call (no cudaMalloc, cudaFree or allocating library routine).  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and caches it.
 * All calls share the one array, which keeps the last call's contents; the error
 * word is cleared by each call.  Calls that overlap on the GPU (different streams
 * or threads at the same time) race on the array and must be serialised by the
 * caller.  RIFT_EINVAL if n < 1 or n > RIFT_NOALLOC_MAX_SAMPLES or a pointer is
 * NULL; RIFT_ENONFINITE if a ln w is NaN or infinite; RIFT_ECUDA on a CUDA error. */
#define RIFT_NOALLOC_MAX_SAMPLES ((int64_t)1 << 31)
int rift_ile_reduce_noalloc(const double *lnw, const double *lnL, int64_t n, double *out, void *cuda_stream);

/* ---- measurement ---------------------------------------------------------------------------
 * Peak rate of a unit the likelihood kernels use, measured on the current device with
 * CUDA events (best of three timed launches after a warm-up), in TFLOP/s: a measurement
 * utility with no counterpart in the paper, so that roofline fractions are taken against
 * this part's rates rather than datasheet figures.
 *   RIFT_PEAK_FP32_FMA     float32 FMA (2 flop), independent chains on every SM;
 *   RIFT_PEAK_TC_F16_N128  tcgen05.mma kind::f16, M = 128, N = 128, K = 16, A in tensor
 *                          memory, float32 accumulation (the likelihood kernel's shape);
 *   RIFT_PEAK_TC_F16_N256  the same with N = 256;
 *   RIFT_PEAK_EX2          ex2.approx.ftz.f32 on the special-function unit, in tera
 *                          operations per second (one exponential counts as one);
 *   RIFT_PEAK_FP64_FMA     float64 FMA (2 flop), independent chains on every SM.
 * The tensor-core runs use one CTA per SM; the tensor-core runs allocate 512 tensor-memory columns per SM, so run
 * them on an otherwise idle device.  Allocates and frees its own small buffers and stream.
 * RIFT_EINVAL for an unknown `what` or a tensor-core rate on a device outside the sm_100
 * family, RIFT_ETIMEOUT if the MMAs did not complete within 2 s, RIFT_ECUDA on a CUDA
 * error. */
#define RIFT_PEAK_FP32_FMA 0
#define RIFT_PEAK_TC_F16_N128 1
#define RIFT_PEAK_TC_F16_N256 2
#define RIFT_PEAK_EX2 3
#define RIFT_PEAK_FP64_FMA 4
int rift_ile_peak_rate(int32_t what, double *tflops);

void rift_ile_destroy(rift_ile_t *h);
const char *rift_ile_strerror(int code);

/* ---- batches of solves -------------------------------------------------------------------
 * Many independent solves (handles with their overlaps set) run as one CUDA graph: each
 * solve's whole adaptive sequence (rift_ile_adapt with its own n_iter and n_per_iter) is
 * a branch with no dependence on the others, so uneven solves share the GPU at once and
 * one graph launch replaces thousands of kernel launches.  The graph is captured on the
 * first run and replayed by later runs; each run continues every solve's adaptive
 * sequence exactly as a rift_ile_adapt call on that handle would (same draws, same
 * results).  The handles must stay alive, and must not be used by other calls while a
 * run is in progress; a handle belongs to at most one batch at a time. */
typedef struct rift_batch rift_batch_t;

/* solves [n] distinct handles (1 <= n <= 65536), n_iter [n], n_per_iter [n] as for
 * rift_ile_adapt; cuda_stream: the stream runs are launched on (NULL: a stream of the
 * batch's own).  RIFT_EINVAL for a bad argument, RIFT_ESTATE if a handle has no
 * overlaps, RIFT_ECUDA if streams or buffers cannot be made. */
int rift_batch_create(rift_ile_t *const *solves, int32_t n, const int32_t *n_iter, const int64_t *n_per_iter,
                      void *cuda_stream, rift_batch_t **out);
/* Run every solve once; out [n] receives each solve's result (status per solve in
 * out[i].status; time_ms[3] of every result is the whole run's device time).  Returns
 * RIFT_OK, or the first failing solve's status. */
int rift_batch_run(rift_batch_t *b, rift_ile_result *out);
/* Kernels one run launches (summed over the solves), or -1 before the first run. */
int64_t rift_batch_kernel_launches(const rift_batch_t *b);
void rift_batch_destroy(rift_batch_t *b);

/* ---- serving ---------------------------------------------------------------------------
 * A request loop that accepts ILE solves (one intrinsic point each: its problem, Q/U/V and
 * sample budget) as they arrive, admits them while the summed device footprint of the
 * solves in flight stays within a budget and a slot is free, and runs admitted solves
 * concurrently, each on its own CUDA stream and host worker, so that requests arriving
 * while others are on the GPU overlap with them (continuous admission, not a queue that
 * drains one solve at a time).  Requests are admitted in arrival order.  Each solve is
 * rift_ile_create -> rift_ile_set_overlaps -> rift_ile_adapt(n_iter, n_per_iter) ->
 * rift_ile_destroy on its slot; its result does not depend on what else is in flight.
 * Times are milliseconds since rift_srv_create (steady clock). */
typedef struct rift_srv rift_srv_t;

typedef struct {
    int64_t hbm_budget_bytes; /* limit on the summed rift_ile_footprint of solves in flight */
    int32_t max_slots;        /* solves in flight at most (1..64)                            */
} rift_srv_config;

typedef struct {
    const rift_ile_config *cfg; /* problem; copied at submit (cfg->max_samples >= n_per_iter) */
    const void *Q, *U, *V;      /* host complex128 arrays, shapes as rift_ile_set_overlaps; copied */
    int32_t n_iter;             /* adaptive iterations (1..RIFT_MAX_ITER)                   */
    int64_t n_per_iter;         /* samples per iteration                                    */
    uint64_t tag;               /* returned with the completion                             */
} rift_srv_request;

typedef struct {
    uint64_t tag;
    int32_t status;            /* RIFT_OK or the first failing call's status */
    rift_ile_result result;
    double t_submit_ms, t_admit_ms, t_done_ms;
} rift_srv_completion;

/* RIFT_EINVAL for a bad configuration; RIFT_ECUDA if no device or stream can be made. */
int rift_srv_create(const rift_srv_config *cfg, rift_srv_t **out);
/* Queue one request (inputs copied before returning).  RIFT_EINVAL for an invalid
 * request; RIFT_ENOMEM if its footprint alone exceeds the budget. */
int rift_srv_submit(rift_srv_t *s, const rift_srv_request *req);
/* Move up to `max` completions into `out` (*n_out of them), waiting up to timeout_ms
 * for the first one (0: do not wait). */
int rift_srv_poll(rift_srv_t *s, rift_srv_completion *out, int32_t max, int32_t timeout_ms, int32_t *n_out);
/* Requests waiting for admission and solves in flight. */
int rift_srv_pending(rift_srv_t *s, int32_t *queued, int32_t *active);
/* Finishes the solves in flight, drops queued requests, joins the workers. */
void rift_srv_destroy(rift_srv_t *s);

#ifdef __cplusplus
}
#endif
#endif /* RIFT_ILE_H */
