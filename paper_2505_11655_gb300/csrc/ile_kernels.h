// Internal launcher interface between the host core and the kernel translation units.
#pragma once

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include <cuda_runtime.h>

#include "ile_common.cuh"

namespace rift {

// Raise a kernel's dynamic shared-memory limit to everything the device allows (less
// its static shared memory), once per kernel and device: every caller sets the same
// value, so concurrent launches from several host threads and streams never race on
// it, and the (slow) attribute calls stay off the launch path.
template <typename Kernel> inline cudaError_t allow_max_dynamic_smem(Kernel kern)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const std::pair<const void *, int> key((const void *)kern, dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(key))
        return cudaSuccess;
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess)
        done.insert(key);
    return e;
}

// Overlaps from frequency-domain inputs (k_precompute.cu): h [M][F], d [K][F] complex,
// w [K][F], f [F] (mirror symmetric), q_t0 [K]; A_scratch [K][M][F]; Q [K][M][n_q],
// U, V [K][M][M] (all device memory).  fft (optional): Q by FFT on the lattice
// f_j = f0 + nidx[j] df, L = f_s / df a power of two (nidx in [0, L)); X, Y [K][M][L] and
// T [L/2] scratch.  *launched (optional): kernels enqueued.
struct FftPlan {
    int L;
    double f0;
    const int *nidx;
    double2 *X, *Y, *T;
};
cudaError_t launch_precompute(const double2 *h, const double2 *d, const double *w, const double *f, int K, int M,
                              int F, const double *q_t0_dev, double fs, int n_q, double2 *A_scratch, double2 *Q,
                              double2 *U, double2 *V, cudaStream_t st, const FftPlan *fft = nullptr,
                              int *launched = nullptr);

// Fair draws (k_fair.cu): fixed-point weights of lnw (max from stats[slot]), their
// running sums, and n_draws sample choices with their time-choice integers.
cudaError_t launch_fair_select(const double *lnw, int64_t n, const double *stats, int slot, uint64_t *W,
                               uint64_t *E, uint64_t *scan_scratch, uint64_t seed, int64_t n_draws,
                               const double *theta, int64_t *idx, double *theta_sel, uint64_t *U_time,
                               cudaStream_t st, int *launched);
// Time bins of m draws from their per-bin ln L rows [m][n_t].
cudaError_t launch_fair_time(const double *lnL_t, int64_t m, int n_t, const uint64_t *U_time, double t_lo,
                             double t_step, int32_t *j_out, double *t_out, cudaStream_t st);

// One bounded mbarrier wait on a barrier nothing completes (k_selftest.cu).
cudaError_t launch_wait_probe(uint64_t limit_ns, int *err, cudaStream_t st);

// Raise the dynamic shared-memory limits of every kernel that needs more than the
// default; called before any launch can be captured into a graph.
cudaError_t prepare_sampler_kernels();
cudaError_t prepare_refine_kernels();
cudaError_t prepare_tile_kernels();
cudaError_t prepare_tc_kernels();
cudaError_t prepare_fix_kernels();

// Per-bin split of j * beta (beta = bin spacing x fs): j*beta = bin_i[j] + bin_f[j], 0 <= bin_f < 1.
struct BinTable {
    const int *bin_i;
    const float *bin_f;
    double ln_nt;   // ln of the number of bins (the uniform time prior's normalisation)
};

// ln L over the time grid for n samples theta[n][6] (float64 everywhere).
//   lnL_tmarg[n] (required), lnL_t[n][n_t] (optional), lnw[i] = lnL_tmarg[i] + lnpw[i] when both given.
cudaError_t launch_lnl_fp64(const Problem &P, const double *theta, int64_t n, double *lnL_tmarg, double *lnL_t,
                            const double *lnpw, double *lnw, int *err, cudaStream_t st);

// Per-sample side outputs of the float32 likelihood kernels (all null, or all set), read
// by the large-term correction: q[i] the float32 template term, m[i] the largest float32
// data term over the time bins, j[i] the first bin of a block of consecutive bins that
// holds the bin of that largest value (the block length is a property of the kernel:
// kPeakBlockTc for the tensor-core tiles, 1 for the CUDA-core tiles).
struct PeakOut {
    float *q = nullptr;
    float *m = nullptr;
    int *j = nullptr;
};
constexpr int kPeakBlockTc = 4;

// Large-term correction of the float32 path (k_fixup.cu).  Mode-pair tables (host-built
// from the mode list) and double-float copies of U, V, Q (built on the device whenever the
// overlaps change).  dmax = 2 max|m|.
struct FixTables {
    const uint16_t *a_ij;   // ordered pairs (a | b << 8) with m_a - m_b = D >= 0, grouped by D
    const int *a_start;     // [dmax + 2] group boundaries
    const uint16_t *b_ij;   // pairs a <= b grouped by S = m_a + m_b
    const int *b_start;     // [2 dmax + 2] group boundaries, by S + dmax
    const float4 *ua;       // [K][nA] U_k,ab (re.hi, re.lo, im.hi, im.lo)
    const float4 *vb;       // [K][nB] (2 - delta_ab) V_k,ab, same layout
    const float4 *qdf;      // [K][M][n_q] Q, same layout
    int nA, nB, dmax;
};
cudaError_t launch_fix_prep(const Problem &P, FixTables T, float4 *ua, float4 *vb, float4 *qdf, cudaStream_t st);
// Lists the samples with po.q + |po.m| > thr (idx, *count; count reset here) and corrects
// their lnL_tmarg (and lnw = lnL_tmarg + lnpw, and the rows of lnL_t, when given) in place.
// blen: the block length of po.j.  *launched: kernels enqueued.
cudaError_t launch_fix(const Problem &P, BinTable bt, FixTables T, const double *theta, int64_t n, PeakOut po,
                       int blen, float thr, uint32_t *idx, uint32_t *count, double *lnL_tmarg, double *lnL_t,
                       const double *lnpw, double *lnw, int *err, cudaStream_t st, int *launched);

// Float32 tiled path.  perm[n] lists sample indices in sky-cell order; outputs are
// written at the original index.  tile_counter: one device int (reset by the launcher).
cudaError_t launch_lnl_fp32(const Problem &P, BinTable bt, const double *theta, const uint32_t *perm, int64_t n,
                            double *lnL_tmarg, double *lnL_t, const double *lnpw, double *lnw, int *err,
                            int *tile_counter, cudaStream_t st, PeakOut po = PeakOut());
size_t lnl_fp32_smem_bytes(const Problem &P);

// Tensor-core variant of the float32 tiled path (tiles of 128 samples, tcgen05 MMA).
bool lnl_tc_fits(const Problem &P, int max_smem);
// Template matrices T_k of the tensor-core kernel from the float64 Gram matrices.
cudaError_t launch_prep_tt(const double2 *U64, const double2 *V64, int K, int M, __half *Ttc, int *tt_exp,
                           cudaStream_t st);
// n_dev (optional): perm holds min(n, *n_dev) entries (a count written on the device);
// n_theta: theta's sample count when perm indexes a larger batch (default n);
// lnl_t_compact: the per-bin output of the sample at position i of perm is row i of lnL_t
// (instead of its sample index's row).
cudaError_t launch_lnl_tc(const Problem &P, BinTable bt, const double *theta, const uint32_t *perm, int64_t n,
                          double *lnL_tmarg, double *lnL_t, const double *lnpw, double *lnw, int *err,
                          int *tile_counter, cudaStream_t st, const uint32_t *n_dev = nullptr,
                          int lnl_t_compact = 0, int64_t n_theta = 0, PeakOut po = PeakOut());
// Builds the float16 hi/lo copy of Q for the tensor-core path.
cudaError_t launch_prep_tc(const double2 *Q64, int K, int M, int n_q, int groups, unsigned int *qmax_bits,
                           __half *Qtc, cudaStream_t st);

// Precision mode RIFT_MIXED: indices of the samples with key[i] >= stats[slot].max - margin
// (idx[*count], ascending), then their float64 re-evaluation in place (lnL_tmarg, and lnw
// when given).  count points to kSelectWords words (the count, then block scratch).
constexpr int kSelectWords = 1 + 1024;
// selected samples whose float32 per-bin values the tiled kernel recomputes for the
// refinement (the rest are recomputed by the refinement itself)
constexpr int64_t kRefineRows = 16384;
cudaError_t launch_select(const double *key, int64_t n, const double *stats, int slot, double margin, uint32_t *idx,
                          uint32_t *count, cudaStream_t st);
// v32 (optional): float32 per-bin ln L of the selected samples, row w for the w-th selected
// sample, for w < v32_rows; the others get their float32 bins recomputed.
cudaError_t launch_refine(const Problem &P, const double *theta, const uint32_t *idx, const uint32_t *count,
                          int64_t max_count, double *lnL_tmarg, const double *lnpw, double *lnw, int *err,
                          cudaStream_t st, const double *v32 = nullptr, int64_t v32_rows = 0);

// Per-sample coefficients: c[n][K][M] (complex), dt[n][K], quad[n]; any may be null.
cudaError_t launch_coeffs(const Problem &P, bool fp64, const double *theta, int64_t n, double2 *c, double *dt,
                          double *quad, cudaStream_t st);

// ---- sampler, sort and reductions ----------------------------------------------------------
struct SamplerDev {
    double *P;       // [6][B] masses
    double *C;       // [6][B+1] running sums
    double *L;       // [6][B] log densities ln(B P[b] / C[B]) of the bins
    int B;
    double d_min, d_max;
    double floor_eps, temper;
    uint64_t seed;
    int marg;        // 1: the distance (dimension 5) is marginalised: no weight, masses kept
};

// Draw n samples of sampler iteration *iter_base + iter_off (the iteration counter is
// read on the device, so a captured graph replays later iterations unchanged).
cudaError_t launch_draw(const SamplerDev &S, const SkyGrid &G, const uint32_t *iter_base, uint32_t iter_off, int64_t n,
                        double *theta, double *lnpw, uint64_t *bins, uint32_t *key, cudaStream_t st);
cudaError_t launch_keys(const SkyGrid &G, const double *theta, int64_t n, uint32_t *key, cudaStream_t st);
// Stable sort of sample indices by sky-cell key (< G.n_cells <= 2^20) into perm: LSD
// radix, 10-bit digits; ties keep index order.  scratch holds sort_scratch_words(n)
// words; *launched (optional) receives the number of kernels enqueued.
constexpr int kRadixBits = 10;
constexpr int kRadixBuckets = 1 << kRadixBits;
size_t sort_scratch_words(int64_t n_max);
// Stable ascending sort of 64-bit keys in place (the low `bits` bits; tmp holds n keys,
// scratch sort64_scratch_words(n) words).
size_t sort64_scratch_words(int64_t n_max);
cudaError_t launch_sort64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, uint32_t *scratch, cudaStream_t st,
                          int *launched = nullptr);
// Exclusive scan of 32-bit counts in place (L < 2^31); scratch holds scan_scratch_words(L).
cudaError_t launch_scan_u32(uint32_t *data, int64_t L, uint32_t *scratch, cudaStream_t st, int *launched = nullptr);
// Exclusive scan of 64-bit counts in place (L < 2^31); scratch holds scan_scratch_words(L).
size_t scan_scratch_words(int64_t L);
cudaError_t launch_scan_u64(uint64_t *data, int64_t L, uint64_t *scratch, cudaStream_t st, int *launched = nullptr);
cudaError_t launch_sort(const SkyGrid &G, const uint32_t *key, int64_t n, uint32_t *scratch, uint32_t *perm,
                        cudaStream_t st, int *launched = nullptr);
// Hilbert-curve grid for a batch of n samples: about `per_cell` samples per cell, at
// least 2^4 and at most 2^kMaxOrder cells a side (host side).
SkyGrid sky_grid_for(int64_t n, int per_cell = 4);

// Reduction of ln w and ln L_tmarg for iteration slot `slot`:
//   stats[slot*8 + 0..7] = lnZ, sigma, n_eff, n_ess, max lnw, max lnL, N, (unused)
//   pooled[0..4] = running max lnw, s1, s2 (relative to the max), N, max lnL over all slots.
// f32_terms: the terms exp(lnw - max) in float32 (relative error ~1e-7, for ln w that carry
// float32 errors themselves: the float32 path); sums, maxima and everything else in float64.
constexpr int kRedBlocks = 304;
cudaError_t launch_reduce(const double *lnw, const double *lnL, int64_t n, double *partial, double *stats, int slot,
                          double *pooled, int reset_pooled, int *err, cudaStream_t st, bool f32_terms = false);
// Histogram adaptation of the sampler from weights exp(beta (lnw - max lnw)) (max from stats[slot]);
// f32_terms as for launch_reduce (the weights stay deterministic: summed exactly in fixed point).
cudaError_t launch_adapt(const SamplerDev &S, const uint64_t *bins, const double *lnw, int64_t n, const double *stats,
                         int slot, uint64_t *hist_partial, cudaStream_t st, bool f32_terms = false);
cudaError_t launch_build_cdf(const SamplerDev &S, cudaStream_t st);
// Final pooled statistics into out[0..7] = lnZ, sigma, n_eff, n_ess, max lnL, N; the
// device iteration counter moves on by `advance`.
cudaError_t launch_pooled_final(const double *pooled, double *out, uint32_t *iter_base, uint32_t advance,
                                cudaStream_t st);

}  // namespace rift
