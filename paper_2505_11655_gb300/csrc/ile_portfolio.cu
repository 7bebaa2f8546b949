// Portfolio integrator on the device (include/rift_ile.h, rift_ile_portfolio):
// arXiv:2505.11655 Sec. IV, "Portfolio integrator".
//
// The sampling prior is the weighted average of two members' priors on the unit cube of
// prior-CDF coordinates: the product-form histogram (the handle's masses, Sec. II B) and
// the adaptive-volume cells (the handle's AV state, Sec. IV A).  One iteration:
//   1. one kernel chooses each draw's member (Philox counter word 3 = 7), draws it with
//      that member's own per-sample draw, and writes ln p - ln p_s of the mixture, the
//      histogram bins of every draw (for the histogram's training) and v (for the AV's);
//   2. the time-marginalised ln L (the same kernels as every other path), the reduction;
//   3. per-member sums of the weights (online maximum, deterministic block order) give
//      each member's n_ESS; the new weights and the freeze rule are decided on the host;
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

// mode 0: the histogram member alone; 1: the AV member alone; 2: both, weights (W0, W1).
__global__ void __launch_bounds__(kPfThreads) portfolio_draw_kernel(
    SamplerDev S, SkyGrid G, const uint64_t *__restrict__ cells, int64_t n_cells, int level, double lnV,
    double invV, double W0, double W1, int mode, uint32_t iter, int64_t n, double *__restrict__ theta,
    double *__restrict__ lnpw, uint64_t *__restrict__ bins, uint32_t *__restrict__ key, double *__restrict__ v_out,
    uint8_t *__restrict__ member)
{
    extern __shared__ double sC[];
    const int B = S.B;
    if (mode != 1)
        hist_load_tables(S, sC);
    __syncthreads();
    const double *sL = sC + 6 * (B + 1) + 6 * B;
    const uint32_t k0 = (uint32_t)S.seed, k1 = (uint32_t)(S.seed >> 32);
    const double d3lo = S.d_min * S.d_min * S.d_min, d3hi = S.d_max * S.d_max * S.d_max;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int m = mode;
        if (mode == 2) {
            const U4 r = philox10(U4{(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, kMemberWord}, k0, k1);
            m = unit53(r.x, r.y) < W0 ? 0 : 1;
        }
        double v[6], th[6], lr;
        uint64_t packed = 0;
        if (m == 0) {
            hist_draw_one(sC, B, 0, iter, i, k0, k1, v, lr, packed);
            hist_theta(v, d3lo, d3hi, th);
            if (mode == 2) {
                const bool in = in_cells(cells, n_cells, av_cell_key(v, level));
                lr = -log(W0 * exp(-lr) + (in ? W1 * invV : 0.0));
            }
        } else {
            av_draw_one(cells, n_cells, level, iter, i, k0, k1, v);
            av_theta(v, d3lo, d3hi, th);
            lr = lnV;
            if (mode == 2) {
                double lnd = 0.0;
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    const int b = min((int)floor(v[d] * (double)B), B - 1);
                    lnd += sL[d * B + b];
                    packed |= (uint64_t)b << (10 * d);
                }
                lr = -log(W0 * exp(lnd) + W1 * invV);
            }
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
        // sky-sort key: the histogram draws' as in its own draw kernel, the AV draws' from theta
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
    __shared__ MAcc sh[2][kPfThreads];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    MAcc a[2] = {{-INFINITY, 0.0, 0.0, 0.0}, {-INFINITY, 0.0, 0.0, 0.0}};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x)
        macc_add(a[member[i] ? 1 : 0], lnw[i]);
    sh[0][threadIdx.x] = a[0];
    sh[1][threadIdx.x] = a[1];
    __syncthreads();
    for (int s = kPfThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] = macc_merge(sh[0][threadIdx.x], sh[0][threadIdx.x + s]);
            sh[1][threadIdx.x] = macc_merge(sh[1][threadIdx.x], sh[1][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) {
        const MAcc r = sh[threadIdx.x][0];
        double *o = partial + 8 * blockIdx.x + 4 * threadIdx.x;
        o[0] = r.mx;
        o[1] = r.s1;
        o[2] = r.s2;
        o[3] = r.cnt;
    }
}

// Pass 2: thread m merges member m's partials in block order into out[m][4].
__global__ void member_sums_final_kernel(const double *__restrict__ partial, int nb, double *__restrict__ out)
{
    const int m = threadIdx.x;
    if (m >= 2)
        return;
    MAcc a{-INFINITY, 0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b) {
        const double *o = partial + 8 * b + 4 * m;
        a = macc_merge(a, MAcc{o[0], o[1], o[2], o[3]});
    }
    out[4 * m] = a.mx;
    out[4 * m + 1] = a.s1;
    out[4 * m + 2] = a.s2;
    out[4 * m + 3] = a.cnt;
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
void floor_weights(const double in[2], const int act[2], double floor, double out[2])
{
    double tot = 0.0;
    for (int a = 0; a < 2; ++a)
        tot += act[a] ? in[a] : 0.0;
    bool fixed[2] = {false, false};
    for (int a = 0; a < 2; ++a)
        out[a] = act[a] ? in[a] / tot : 0.0;
    for (;;) {
        bool any = false;
        for (int a = 0; a < 2; ++a)
            if (act[a] && !fixed[a] && out[a] < floor)
                fixed[a] = any = true;
        if (!any)
            return;
        int n_fixed = 0;
        double free_sum = 0.0;
        for (int a = 0; a < 2; ++a) {
            if (fixed[a]) {
                out[a] = floor;
                ++n_fixed;
            } else if (act[a]) {
                free_sum += out[a];
            }
        }
        const double scale = (1.0 - floor * n_fixed) / free_sum;
        for (int a = 0; a < 2; ++a)
            if (act[a] && !fixed[a])
                out[a] *= scale;
    }
}

int pf_alloc(rift_ile_t *h)
{
    auto &p = h->pf;
    const int64_t N = h->cap;
    int rc;
    if ((rc = dalloc(h, &p.member, (size_t)N)) || (rc = dalloc(h, &p.v, (size_t)N * 6)) ||
        (rc = dalloc(h, &p.v_av, (size_t)N * 6)) || (rc = dalloc(h, &p.lnL_av, (size_t)N)) ||
        (rc = dalloc(h, &p.part, (size_t)8 * kPfSumBlocks)) || (rc = dalloc(h, &p.sums, (size_t)8)))
        return rc;
    CK(allow_max_dynamic_smem(portfolio_draw_kernel));
    p.alloc = true;
    return RIFT_OK;
}

int pf_restart(rift_ile_t *h, bool with_av)
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
    return RIFT_OK;
}

int portfolio_iteration(rift_ile_t *h, int64_t n, int slot, bool reset_pooled, const rift_portfolio_config &cfg)
{
    auto &a = h->av;
    auto &p = h->pf;
    cudaStream_t st = h->stream;
    const uint32_t g = p.iter;
    const bool has_av = (cfg.members & RIFT_MEMBER_AV) != 0;
    const int act[2] = {(cfg.members & RIFT_MEMBER_HIST) ? 1 : 0, has_av && (int64_t)g >= cfg.av_start ? 1 : 0};
    if (!p.have_w || (has_av && cfg.av_start > 0 && (int64_t)g == cfg.av_start)) {
        floor_weights(cfg.w_init, act, 0.0, p.W);
        p.have_w = true;
    }
    const int mode = act[0] && act[1] ? 2 : act[0] ? 0 : 1;
    const double W[2] = {p.W[0], p.W[1]};
    SamplerDev S = sampler_of(h);
    RK(grid_for_batch(h, n));
    // 1. member choice and draws
    CK(mark(h, slot, 0));
    const size_t smem = mode == 1 ? 0 : sizeof(double) * hist_table_doubles(S.B);
    portfolio_draw_kernel<<<grid_n(n), kPfThreads, smem, st>>>(
        S, h->grid, a.cells, a.n_cells, a.level, has_av ? std::log(a.V) : 0.0, has_av ? 1.0 / a.V : 0.0, W[0], W[1],
        mode, g, n, h->theta, h->lnpw, h->bins, h->key, p.v, p.member);
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
    // 3. per-member n_ESS and the new weights
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kPfSumBlocks, (n + kPfThreads - 1) / kPfThreads));
    member_sums_kernel<<<nb, kPfThreads, 0, st>>>(h->lnw, p.member, n, p.part);
    member_sums_final_kernel<<<1, 32, 0, st>>>(p.part, nb, p.sums);
    h->launches += 1 + sorted + 1 + 2 + 2;
    double sums[8];
    CK(cudaMemcpyAsync(sums, p.sums, sizeof(sums), cudaMemcpyDeviceToHost, st));
    RK(sync_and_err(h));
    double ess[2];
    int64_t cnt[2];
    for (int m = 0; m < 2; ++m) {
        cnt[m] = (int64_t)sums[4 * m + 3];
        ess[m] = act[m] && sums[4 * m + 2] > 0.0 ? sums[4 * m + 1] * sums[4 * m + 1] / sums[4 * m + 2] : 0.0;
    }
    double W_next[2] = {W[0], W[1]};
    if (cfg.adapt_weights && mode == 2 && ess[0] + ess[1] > 0.0)
        floor_weights(ess, act, kWeightFloor / 2.0, W_next);
    const int frozen[2] = {!act[0] || W_next[0] < kFreezeBelow ? 1 : 0, !act[1] || W_next[1] < kFreezeBelow ? 1 : 0};
    // 4. training
    if (!frozen[0]) {
        CK(launch_adapt(S, h->bins, h->lnw, n, h->stats, slot, h->hist_partial, st, f32_terms));
        h->launches += 2;
    }
    if (!frozen[1] && cnt[1] > 0) {
        if (mode == 1) {
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
    CK(mark(h, slot, 3));
    for (int m = 0; m < 2; ++m) {
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
    if (!h || !cfg || h->cfg.distance_marg || n_iter < 1 || n_iter > RIFT_MAX_ITER || n_per_iter < 1 ||
        n_per_iter > h->cap || cfg->members < 1 || cfg->members > (RIFT_MEMBER_HIST | RIFT_MEMBER_AV) ||
        cfg->av_start < 0 || (cfg->members == RIFT_MEMBER_AV && cfg->av_start != 0) ||
        (cfg->adapt_weights != 0 && cfg->adapt_weights != 1))
        return RIFT_EINVAL;
    for (int m = 0; m < 2; ++m)
        if ((cfg->members >> m) & 1)
            if (!(cfg->w_init[m] > 0.0) || !std::isfinite(cfg->w_init[m]))
                return RIFT_EINVAL;
    const bool has_av = (cfg->members & RIFT_MEMBER_AV) != 0;
    if (has_av && (!(cfg->p_thr > 0.0) || !(cfg->p_thr <= 1.0) || cfg->n_min_star < 1 || cfg->capacity < n_per_iter ||
                   cfg->capacity > ((int64_t)1 << 31) - 2 || (h->av.cap != 0 && h->av.cap != cfg->capacity)))
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    bool fresh = restart != 0 || !h->pf.alloc;
    if (!h->pf.alloc)
        RK(pf_alloc(h));
    if (has_av && h->av.cap == 0) {
        RK(av_alloc(h, cfg->capacity));
        RK(av_restart(h));
    }
    if (fresh)
        RK(pf_restart(h, has_av));
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
    for (int m = 0; m < 2; ++m) {
        info->active[m] = p.active[m];
        info->frozen[m] = p.frozen[m];
        info->W_last[m] = p.W_last[m];
        info->W_next[m] = p.W[m];
        info->n_ess[m] = p.n_ess[m];
        info->n_drawn[m] = p.n_drawn[m];
    }
    return RIFT_OK;
}

}  // extern "C"
