// Host core of the ILE library: configuration checks, device buffers, the order of
// kernel launches for each entry point of include/rift_ile.h, and result assembly.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "ile_handle.h"

using namespace rift;

namespace {

constexpr uint64_t kStateMagic = 0x31454C4954464952ull;   // "RIFTILE1"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
    uint64_t magic;
    uint32_t version;
    uint32_t n_bins;
    uint64_t seed;
    uint32_t iteration;
    uint32_t reserved;
};

// Q window padding of the float32 planes: one chunk window past the end.
constexpr int kQPad = 256 + 16;

}  // namespace


namespace rift {
namespace host {

// Device buffers come from the device's stream-ordered memory pool on the handle's
// stream: no device-wide synchronisation, and freed blocks stay cached for the next
// handle (the pool's release threshold is raised once per process).
void keep_pool_cached()
{
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    });
}

void release(rift_ile_t *h)
{
    if (!h)
        return;
    if (h->graph)
        cudaGraphExecDestroy(h->graph);
    for (void *p : h->allocs)
        cudaFreeAsync(p, h->stream);
    h->allocs.clear();
    cudaStreamSynchronize(h->stream);
    for (auto &row : h->ev)
        for (auto &e : row)
            cudaEventDestroy(e);
    if (h->own_stream)
        cudaStreamDestroy(h->stream);
    cudaGetLastError();
    delete h;
}

int ensure_events(rift_ile_t *h, int n)
{
    while ((int)h->ev.size() < n) {
        std::array<cudaEvent_t, 4> row{};
        for (auto &e : row)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return RIFT_ECUDA;
            }
        h->ev.push_back(row);
    }
    return RIFT_OK;
}

double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i)
        r *= i;
    return r;
}

// Wigner small-d d^l_{m',2}(beta) written as a sum over s of
//   (-1)^(m'-2+s) sqrt((l+m')!(l-m')!(l+2)!(l-2)!) / ((l+2-s)! s! (m'-2+s)! (l-m'-s)!)
//   cos(beta/2)^(2l+2-m'-2s) sin(beta/2)^(m'-2+2s),
// so that -2Y_lm(beta, .) = sqrt((2l+1)/4pi) d^l_{m,2}(beta) e^{i m .}.
int wigner_table(int l, int m, double *coef, int8_t *pc, int8_t *ps)
{
    const double norm = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi));
    const double root = std::sqrt(factorial(l + m) * factorial(l - m) * factorial(l + 2) * factorial(l - 2));
    int s0 = std::max(0, 2 - m), s1 = std::min(l + 2, l - m);
    int nt = 0;
    for (int s = s0; s <= s1; ++s) {
        int sign_exp = m - 2 + s;
        double sign = (std::abs(sign_exp) % 2) ? -1.0 : 1.0;
        double v = sign * root / (factorial(l + 2 - s) * factorial(s) * factorial(m - 2 + s) * factorial(l - m - s));
        if (nt >= kMaxWTerms)
            return -1;
        coef[nt] = norm * v;
        pc[nt] = (int8_t)(2 * l + 2 - m - 2 * s);
        ps[nt] = (int8_t)(m - 2 + 2 * s);
        ++nt;
    }
    return nt;
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n from the
// three-term recurrence, starting at the Chebyshev-like guesses cos(pi (i + 3/4) / (n + 1/2)).
void gauss_legendre(int n, double *t, double *w)
{
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16)
                break;
        }
        t[n - 1 - i] = x;   // ascending
        w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

int map_err(int flags)
{
    if (flags & kErrTimeout)
        return RIFT_ETIMEOUT;
    if (flags & kErrRange)
        return RIFT_ERANGE;
    if (flags & kErrNonFinite)
        return RIFT_ENONFINITE;
    return RIFT_OK;
}


SamplerDev sampler_of(const rift_ile_t *h)
{
    SamplerDev S;
    S.P = h->P;
    S.C = h->C;
    S.L = h->Lg;
    S.B = h->cfg.n_bins;
    S.d_min = h->cfg.d_min_mpc;
    S.d_max = h->cfg.d_max_mpc;
    S.floor_eps = h->cfg.adapt_floor;
    S.temper = h->cfg.adapt_temper;
    S.seed = h->cfg.seed;
    S.marg = h->cfg.distance_marg;
    return S;
}

int validate(const rift_ile_config *c)
{
    if (!c || c->n_det < 1 || c->n_det > RIFT_MAX_DET || c->n_modes < 1 || c->n_modes > RIFT_MAX_MODES)
        return RIFT_EINVAL;
    if (c->distance_marg != 0 && c->distance_marg != 1)
        return RIFT_EINVAL;
    if (!c->det_tensor || !c->det_pos_m || !c->lm || !c->q_t0_s)
        return RIFT_EINVAL;
    if (!(c->fs_hz > 0) || c->n_q < 2 || c->n_t < 1 || !(c->t_hi_s >= c->t_lo_s))
        return RIFT_EINVAL;
    if (!(c->d_ref_mpc > 0) || !(c->d_min_mpc > 0) || !(c->d_max_mpc > c->d_min_mpc))
        return RIFT_EINVAL;
    if (c->quad_norm != RIFT_QUAD_QUARTER && c->quad_norm != RIFT_QUAD_HALF)
        return RIFT_EINVAL;
    if (c->precision != RIFT_FP64 && c->precision != RIFT_FP32 && c->precision != RIFT_MIXED)
        return RIFT_EINVAL;
    if (c->n_bins < 2 || c->n_bins > RIFT_MAX_BINS || !(c->adapt_floor >= 0 && c->adapt_floor < 1) ||
        !(c->adapt_temper > 0))
        return RIFT_EINVAL;
    if (c->max_samples < 1 || c->max_samples > (int64_t)0x7fffffff)
        return RIFT_EINVAL;
    std::set<std::pair<int, int>> seen;
    for (int i = 0; i < c->n_modes; ++i) {
        int l = c->lm[2 * i], m = c->lm[2 * i + 1];
        if (l < 2 || l > kMaxL || m < -l || m > l || !seen.insert({l, m}).second)
            return RIFT_EINVAL;
    }
    for (int k = 0; k < c->n_det; ++k) {
        for (int i = 0; i < 9; ++i)
            if (!std::isfinite(c->det_tensor[9 * k + i]))
                return RIFT_EINVAL;
        double r = 0;
        for (int i = 0; i < 3; ++i) {
            if (!std::isfinite(c->det_pos_m[3 * k + i]))
                return RIFT_EINVAL;
            r += c->det_pos_m[3 * k + i] * c->det_pos_m[3 * k + i];
        }
        double rc = std::sqrt(r) / kC;
        double umin = (c->t_lo_s - rc - c->q_t0_s[k]) * c->fs_hz;
        double umax = (c->t_hi_s + rc - c->q_t0_s[k]) * c->fs_hz;
        if (!(umin >= 1e-3) || !(umax <= (double)(c->n_q - 2) - 1e-3))
            return RIFT_ERANGE;
    }
    return RIFT_OK;
}

// Builds float32 planes and Gram copies from the float64 device copies; flags NaN/Inf.
__global__ void prep_overlaps_kernel(const double2 *__restrict__ Q64, const double2 *__restrict__ U64,
                                     const double2 *__restrict__ V64, int K, int M, int n_q, int n_q_pad,
                                     float *__restrict__ Qr32, float2 *__restrict__ U32, float2 *__restrict__ V32,
                                     int *err)
{
    const int64_t total = (int64_t)K * 2 * M * n_q_pad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = e / n_q_pad;
        int c = (int)(e - row * n_q_pad);
        int k = (int)(row / (2 * M)), r = (int)(row % (2 * M));
        float v = 0.f;
        if (c < n_q) {
            double2 q = Q64[((int64_t)k * M + r / 2) * n_q + c];
            double x = (r & 1) ? q.y : q.x;
            if (!isfinite(x))
                atomicOr(err, kErrNonFinite);
            v = (float)x;
        }
        Qr32[e] = v;
    }
    const int64_t g = (int64_t)K * M * M;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g; e += (int64_t)gridDim.x * blockDim.x) {
        double2 u = U64[e], v = V64[e];
        if (!isfinite(u.x) || !isfinite(u.y) || !isfinite(v.x) || !isfinite(v.y))
            atomicOr(err, kErrNonFinite);
        U32[e] = make_float2((float)u.x, (float)u.y);
        V32[e] = make_float2((float)v.x, (float)v.y);
    }
}

int sync_and_err(rift_ile_t *h, int *flags_out)
{
    int flags = 0;
    CK(cudaMemcpyAsync(&h->host_out[0], h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(&flags, &h->host_out[0], sizeof(int));
    if (flags_out)
        *flags_out = flags;
    return map_err(flags);
}

bool use_fp32(const rift_ile_t *h) { return h->cfg.precision != RIFT_FP64; }

// Without a tuned plan: tensor-core tiles pay off once a batch fills the sky densely
// enough that 128 samples share a 128-column Q window.
constexpr int64_t kTcMinBatch = 100000;

bool use_tc(const rift_ile_t *h, int64_t n)
{
    if (!h->tc_ok || h->tc_mode == 0)
        return false;
    if (h->tc_mode == 1)
        return true;
    return h->plan.tc >= 0 ? h->plan.tc == 1 : n >= kTcMinBatch;
}

cudaError_t launch_tiled(rift_ile_t *h, const double *theta, int64_t n, double *lnL_tmarg, double *lnL_t,
                         const double *lnpw, double *lnw)
{
    const BinTable bt{h->bin_i, h->bin_f, std::log((double)h->prob.n_t)};
    PeakOut po;
    if (h->fix_on) {
        po.q = h->aux_q;
        po.m = h->aux_m;
        po.j = h->aux_j;
    }
    const bool tc = use_tc(h, n);
    cudaError_t e = tc ? launch_lnl_tc(h->prob, bt, theta, h->perm, n, lnL_tmarg, lnL_t, lnpw, lnw, h->err,
                                       h->tile_counter, h->stream, nullptr, 0, 0, po)
                       : launch_lnl_fp32(h->prob, bt, theta, h->perm, n, lnL_tmarg, lnL_t, lnpw, lnw, h->err,
                                         h->tile_counter, h->stream, po);
    if (e != cudaSuccess || !h->fix_on)
        return e;
    // the samples whose float32 terms are large enough for their rounding to reach the
    // parity bar: template term and peak data term again in double-float
    int k = 0;
    e = launch_fix(h->prob, bt, h->fix, theta, n, po, tc ? kPeakBlockTc : 1, h->fix_thr, h->fix_idx, h->fix_count,
                   lnL_tmarg, lnL_t, lnpw, lnw, h->err, h->stream, &k);
    h->launches += k;
    return e;
}

// RIFT_MIXED: samples whose log-weight is within kMixedMargin of the batch maximum
// are re-evaluated in float64 (their weight relative to the largest is >= e^-40).
constexpr double kMixedMargin = 40.0;
// the float32 modes correct every sample whose template term plus largest data term
// exceeds this (k_fixup.cu)
constexpr float kFixThreshold = 600.f;

int refine_batch(rift_ile_t *h, const double *theta, int64_t n, double *lnL_tmarg, const double *lnpw, double *lnw)
{
    const double *key = lnw ? lnw : lnL_tmarg;
    CK(launch_reduce(key, lnL_tmarg, n, h->red_partial, h->stats, kScratchSlot, h->pooled_scratch, 1, h->err,
                     h->stream));
    CK(launch_select(key, n, h->stats, kScratchSlot, kMixedMargin, h->sel_idx, h->sel_count, h->stream));
    // the tensor-core kernel recomputes the float32 per-bin ln L of the first refine_rows
    // selected samples (a few tiles), so the refinement itself evaluates only the bins
    // within its margin in float64
    int64_t rows = 0;
    if (h->refine_bins && use_tc(h, n)) {
        const BinTable bt{h->bin_i, h->bin_f, std::log((double)h->prob.n_t)};
        rows = std::min<int64_t>(h->refine_rows, n);
        CK(launch_lnl_tc(h->prob, bt, theta, h->sel_idx, rows, lnL_tmarg, h->refine_bins, lnpw, lnw, h->err,
                         h->tile_counter, h->stream, h->sel_count, 1, n));
        h->launches += 1;
    }
    CK(launch_refine(h->prob, theta, h->sel_idx, h->sel_count, n, lnL_tmarg, lnpw, lnw, h->err, h->stream,
                     h->refine_bins, rows));
    h->launches += 6;
    return RIFT_OK;
}

// Sky grid sized for a batch of n samples.
int grid_for_batch(rift_ile_t *h, int64_t n)
{
    SkyGrid g = sky_grid_for(n, h->plan.per_cell);
    const Problem &P = h->prob;
    const bool delay3 = P.K >= 3 && h->plan.delay3;
    if (P.K <= 2 || delay3) {
        g.mode = P.K == 1 ? kSortDelay1 : P.K == 2 ? kSortDelay2 : kSortDelay3;
        if (delay3) {   // as many cells as the sky grid, 8 per level of three delays
            g.order = std::max(1, 2 * g.order / 3);
            g.n_cells = 1 << (3 * g.order);
        }
        g.gmst = P.gmst;
        for (int k = 0; k < std::min(P.K, 3); ++k) {
            double r2 = 0.0;
            for (int i = 0; i < 3; ++i) {
                g.x[k][i] = P.xpos[k][i];
                r2 += P.xpos[k][i] * P.xpos[k][i];
            }
            g.span[k] = std::sqrt(r2);
        }
    }
    h->grid = g;
    return RIFT_OK;
}

// Stage timer: inside a graph capture the record becomes an event node, so replays
// time themselves.
cudaError_t mark(rift_ile_t *h, int slot, int stage)
{
    if (!h->timed)
        return cudaSuccess;
    if (h->capturing)
        return cudaEventRecordWithFlags(h->ev[slot][stage], h->stream, cudaEventRecordExternal);
    return cudaEventRecord(h->ev[slot][stage], h->stream);
}

// ln L for n device-resident samples (theta [n][6]); perm/key scratch from the handle.
int eval_device(rift_ile_t *h, const double *theta, int64_t n, double *lnL_tmarg, double *lnL_t, const double *lnpw,
                double *lnw)
{
    if (!use_fp32(h)) {
        CK(launch_lnl_fp64(h->prob, theta, n, lnL_tmarg, lnL_t, lnpw, lnw, h->err, h->stream));
        h->launches += 1;
        return RIFT_OK;
    }
    RK(choose_plan(h, n, false));
    RK(grid_for_batch(h, n));
    int sorted = 0;
    CK(launch_keys(h->grid, theta, n, h->key, h->stream));
    CK(launch_sort(h->grid, h->key, n, h->sort_scratch, h->perm, h->stream, &sorted));
    h->launches += 2 + sorted;   // keys, sort, tiled likelihood
    CK(launch_tiled(h, theta, n, lnL_tmarg, lnL_t, lnpw, lnw));
    if (h->cfg.precision == RIFT_MIXED)
        RK(refine_batch(h, theta, n, lnL_tmarg, lnpw, lnw));
    return RIFT_OK;
}

// One draw -> sort -> likelihood -> reduce (-> adapt) iteration into stats slot `slot`;
// the draw uses sampler iteration (device counter + slot).
int run_iteration(rift_ile_t *h, int64_t n, int slot, bool adapt, bool reset_pooled)
{
    SamplerDev S = sampler_of(h);
    RK(grid_for_batch(h, n));
    CK(mark(h, slot, 0));
    CK(launch_draw(S, h->grid, h->iter_dev, (uint32_t)slot, n, h->theta, h->lnpw, h->bins, h->key, h->stream));
    int sorted = 0;
    if (use_fp32(h))
        CK(launch_sort(h->grid, h->key, n, h->sort_scratch, h->perm, h->stream, &sorted));
    CK(mark(h, slot, 1));
    if (!use_fp32(h)) {
        CK(launch_lnl_fp64(h->prob, h->theta, n, h->lnL, nullptr, h->lnpw, h->lnw, h->err, h->stream));
    } else {
        CK(launch_tiled(h, h->theta, n, h->lnL, nullptr, h->lnpw, h->lnw));
        if (h->cfg.precision == RIFT_MIXED)
            RK(refine_batch(h, h->theta, n, h->lnL, h->lnpw, h->lnw));
    }
    CK(mark(h, slot, 2));
    const bool f32_terms = h->cfg.precision == RIFT_FP32;
    CK(launch_reduce(h->lnw, h->lnL, n, h->red_partial, h->stats, slot, h->pooled, reset_pooled ? 1 : 0, h->err,
                     h->stream, f32_terms));
    if (adapt)
        CK(launch_adapt(S, h->bins, h->lnw, n, h->stats, slot, h->hist_partial, h->stream, f32_terms));
    CK(mark(h, slot, 3));
    h->launches += 1 + sorted + 1 + 2 + (adapt ? 2 : 0);
    return RIFT_OK;
}

int enqueue_adapt(rift_ile_t *h, int32_t n_iter, int64_t n)
{
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    for (int g = 0; g < n_iter; ++g)
        RK(run_iteration(h, n, g, true, g == 0));
    CK(launch_pooled_final(h->pooled, h->final_out, h->iter_dev, (uint32_t)n_iter, h->stream));
    h->launches += 1;
    return RIFT_OK;
}

int collect_result(rift_ile_t *h, int n_iter, rift_ile_result *out)
{
    // host_out layout: [0] err word, [1..8) final, [8..) stats
    CK(cudaMemcpyAsync(&h->host_out[1], h->final_out, sizeof(double) * 6, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&h->host_out[8], h->stats, sizeof(double) * 8 * n_iter, cudaMemcpyDeviceToHost, h->stream));
    int flags = 0;
    int rc = sync_and_err(h, &flags);
    if (!out)
        return rc;
    std::memset(out, 0, sizeof(*out));
    const double *f = &h->host_out[1];
    out->lnZ = f[0];
    out->sigma_lnZ = f[1];
    out->n_eff = f[2];
    out->n_ess = f[3];
    out->lnL_max = f[4];
    out->n_total = (int64_t)f[5];
    out->n_iter = n_iter;
    out->status = rc;
    for (int g = 0; g < n_iter; ++g) {
        const double *s = &h->host_out[8 + 8 * g];
        out->lnZ_iter[g] = s[0];
        out->sigma_iter[g] = s[1];
        out->n_eff_iter[g] = s[2];
        out->n_ess_iter[g] = s[3];
        if (!h->timed)
            continue;
        float a = 0, b = 0, c = 0, d = 0;
        cudaEventElapsedTime(&a, h->ev[g][0], h->ev[g][1]);
        cudaEventElapsedTime(&b, h->ev[g][1], h->ev[g][2]);
        cudaEventElapsedTime(&c, h->ev[g][2], h->ev[g][3]);
        cudaEventElapsedTime(&d, h->ev[g][0], h->ev[g][3]);
        out->time_ms[0] += a;
        out->time_ms[1] += b;
        out->time_ms[2] += c;
        out->time_ms[3] += d;
    }
    cudaGetLastError();
    return rc;
}

bool graphs_enabled()
{
    const char *env = std::getenv("RIFT_ILE_GRAPHS");
    return !(env && env[0] == '0');
}

void drop_graph(rift_ile_t *h)
{
    if (h->graph)
        cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_iter = 0;
    h->graph_n = 0;
}

// Capture enqueue_adapt(n_iter, n) on the handle's stream into h->graph.
int capture_adapt(rift_ile_t *h, int32_t n_iter, int64_t n)
{
    drop_graph(h);
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = h->launches;
    h->capturing = true;
    int rc = enqueue_adapt(h, n_iter, n);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    const int64_t per_run = h->launches - l0;
    h->launches = l0;
    if (rc != RIFT_OK || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != RIFT_OK ? rc : RIFT_ECUDA;
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    h->graph_iter = n_iter;
    h->graph_n = n;
    h->graph_plan = h->plan;
    h->graph_launches = per_run;
    return RIFT_OK;
}

}  // namespace host
}  // namespace rift

using namespace rift::host;

// ============================================================================ ABI

extern "C" {

const char *rift_ile_strerror(int code)
{
    switch (code) {
    case RIFT_OK: return "ok";
    case RIFT_EINVAL: return "invalid argument";
    case RIFT_ENOMEM: return "out of memory";
    case RIFT_ECUDA: return "CUDA error";
    case RIFT_ERANGE: return "time-shifted Q index outside the Q window";
    case RIFT_ENONFINITE: return "non-finite value in inputs or results";
    case RIFT_ETIMEOUT: return "bounded device wait timed out";
    case RIFT_ESTATE: return "call out of order or malformed state";
    default: return "unknown status";
    }
}

int rift_ile_create(const rift_ile_config *cfg, void *cuda_stream, rift_ile_t **out)
{
    if (!out)
        return RIFT_EINVAL;
    *out = nullptr;
    int v = validate(cfg);
    if (v != RIFT_OK)
        return v;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    keep_pool_cached();
    rift_ile_t *h = new (std::nothrow) rift_ile_t();
    if (!h)
        return RIFT_ENOMEM;
    h->cfg = *cfg;
    const int K = cfg->n_det, M = cfg->n_modes;
    h->det_tensor.assign(cfg->det_tensor, cfg->det_tensor + 9 * K);
    h->det_pos.assign(cfg->det_pos_m, cfg->det_pos_m + 3 * K);
    h->q_t0.assign(cfg->q_t0_s, cfg->q_t0_s + K);
    h->lm.assign(cfg->lm, cfg->lm + 2 * M);
    h->cfg.det_tensor = h->det_tensor.data();
    h->cfg.det_pos_m = h->det_pos.data();
    h->cfg.q_t0_s = h->q_t0.data();
    h->cfg.lm = h->lm.data();
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!h->stream) {
        // a stream of the handle's own (blocking: ordered with the legacy default
        // stream), so that repeated adaptive sequences can be captured as graphs
        if (cudaStreamCreate(&h->stream) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return RIFT_ECUDA;
        }
        h->own_stream = true;
    }
    h->cap = cfg->max_samples;

    Problem &P = h->prob;
    P.K = K;
    P.M = M;
    P.n_q = cfg->n_q;
    P.n_t = cfg->n_t;
    P.n_q_pad = ((cfg->n_q + 3) & ~3) + kQPad;
    P.fs = cfg->fs_hz;
    P.t_lo = cfg->t_lo_s;
    P.t_step = cfg->n_t > 1 ? (cfg->t_hi_s - cfg->t_lo_s) / (cfg->n_t - 1) : 0.0;
    P.gmst = cfg->gmst_rad;
    P.d_ref = cfg->d_ref_mpc;
    P.kappa = cfg->quad_norm == RIFT_QUAD_HALF ? 0.5 : 0.25;
    P.dist_marg = cfg->distance_marg;
    P.dm_xlo = cfg->d_ref_mpc / cfg->d_max_mpc;
    P.dm_xhi = cfg->d_ref_mpc / cfg->d_min_mpc;
    P.dm_lnC = std::log(3.0 * cfg->d_ref_mpc * cfg->d_ref_mpc * cfg->d_ref_mpc /
                        (cfg->d_max_mpc * cfg->d_max_mpc * cfg->d_max_mpc -
                         cfg->d_min_mpc * cfg->d_min_mpc * cfg->d_min_mpc));
    P.dm_lnub = P.dm_lnC + std::log((1.0 / (P.dm_xlo * P.dm_xlo * P.dm_xlo) -
                                     1.0 / (P.dm_xhi * P.dm_xhi * P.dm_xhi)) / 3.0);
    gauss_legendre(16, P.gl16_t, P.gl16_w);
    {
        double t10[10], w10[10];
        gauss_legendre(10, t10, w10);
        for (int i = 0; i < 10; ++i) {
            P.gl10_tf[i] = (float)t10[i];
            P.gl10_wf[i] = (float)w10[i];
        }
    }
    P.dm_xlo_f = (float)P.dm_xlo;
    P.dm_xhi_f = (float)P.dm_xhi;
    P.dm_lnC_f = (float)P.dm_lnC;
    P.dm_lnub_f = (float)P.dm_lnub;
    for (int k = 0; k < K; ++k) {
        const double *D = cfg->det_tensor + 9 * k;
        P.Dten[k][0] = D[0];
        P.Dten[k][1] = D[4];
        P.Dten[k][2] = D[8];
        P.Dten[k][3] = 0.5 * (D[1] + D[3]);
        P.Dten[k][4] = 0.5 * (D[2] + D[6]);
        P.Dten[k][5] = 0.5 * (D[5] + D[7]);
        for (int i = 0; i < 6; ++i)
            P.Dten_f[k][i] = (float)P.Dten[k][i];
        for (int i = 0; i < 3; ++i)
            P.xpos[k][i] = cfg->det_pos_m[3 * k + i] / kC;
        P.q_t0[k] = cfg->q_t0_s[k];
        P.ufs0[k] = (P.t_lo - P.q_t0[k]) * P.fs;
        for (int i = 0; i < 3; ++i)
            P.xfs[k][i] = -P.xpos[k][i] * P.fs;
    }
    for (int m = 0; m < M; ++m) {
        P.mode_m[m] = cfg->lm[2 * m + 1];
        int nt = wigner_table(cfg->lm[2 * m], cfg->lm[2 * m + 1], P.wcoef[m], P.wpc[m], P.wps[m]);
        if (nt < 0) {
            release(h);
            return RIFT_EINVAL;
        }
        P.wn[m] = (int8_t)nt;
        for (int t = 0; t < nt; ++t)
            P.wcoef_f[m][t] = (float)P.wcoef[m][t];
    }

    int rc = RIFT_OK;
    const int64_t N = h->cap;
    const int B = cfg->n_bins;
    if ((rc = dalloc(h, &h->Q64, (size_t)K * M * cfg->n_q)) || (rc = dalloc(h, &h->U64, (size_t)K * M * M)) ||
        (rc = dalloc(h, &h->V64, (size_t)K * M * M)) || (rc = dalloc(h, &h->Qr32, (size_t)K * 2 * M * P.n_q_pad)) ||
        (rc = dalloc(h, &h->U32, (size_t)K * M * M)) || (rc = dalloc(h, &h->V32, (size_t)K * M * M)) ||
        (rc = dalloc(h, &h->Ttc, (size_t)K * 2 * ((2 * M + 15) / 16 * 16) * ((2 * M + 15) / 16 * 16))) ||
        (rc = dalloc(h, &h->tt_exp, (size_t)K)) ||
        (rc = dalloc(h, &h->bin_i, (size_t)cfg->n_t)) || (rc = dalloc(h, &h->bin_f, (size_t)cfg->n_t)) ||
        (rc = dalloc(h, &h->theta, (size_t)N * 6)) || (rc = dalloc(h, &h->lnpw, (size_t)N)) ||
        (rc = dalloc(h, &h->lnL, (size_t)N)) || (rc = dalloc(h, &h->lnw, (size_t)N)) ||
        (rc = dalloc(h, &h->bins, (size_t)N)) || (rc = dalloc(h, &h->key, (size_t)N)) ||
        (rc = dalloc(h, &h->perm, (size_t)N)) || (rc = dalloc(h, &h->sort_scratch, sort_scratch_words(N))) ||
        (rc = dalloc(h, &h->tile_counter, (size_t)4)) ||
        (rc = dalloc(h, &h->qmax_bits, (size_t)4)) ||
        (rc = dalloc(h, &h->Qtc, (size_t)K * 2 * ((cfg->n_q + 7) / 8 + 17) * ((2 * M + 15) / 16 * 16) * 8)) ||
        (rc = dalloc(h, &h->red_partial, (size_t)5 * kRedBlocks)) ||
        (rc = dalloc(h, &h->hist_partial, (size_t)152 * 12 * B)) ||
        (rc = dalloc(h, &h->stats, (size_t)8 * (RIFT_MAX_ITER + 1))) || (rc = dalloc(h, &h->pooled, (size_t)8)) ||
        (rc = dalloc(h, &h->pooled_scratch, (size_t)8)) || (rc = dalloc(h, &h->sel_idx, (size_t)N)) ||
        (rc = dalloc(h, &h->sel_count, (size_t)kSelectWords)) ||
        (rc = dalloc(h, &h->final_out, (size_t)8)) || (rc = dalloc(h, &h->P, (size_t)6 * B)) ||
        (rc = dalloc(h, &h->C, (size_t)6 * (B + 1))) || (rc = dalloc(h, &h->Lg, (size_t)6 * B)) || (rc = dalloc(h, &h->err, (size_t)4)) ||
        (rc = dalloc(h, &h->iter_dev, (size_t)4))) {
        release(h);
        return rc;
    }
    // the large-term correction runs in the float32 modes (not with the distance marginal,
    // whose per-bin values are no difference of two large terms)
    h->fix_on = cfg->precision != RIFT_FP64 && !cfg->distance_marg;
    if (h->fix_on) {
        // mode-pair tables, grouped by m_a - m_b >= 0 (ordered pairs) and by m_a + m_b (a <= b)
        int mmax = 0;
        for (int m = 0; m < M; ++m)
            mmax = std::max(mmax, std::abs(cfg->lm[2 * m + 1]));
        const int dmax = 2 * mmax;
        std::vector<uint16_t> aij, bij;
        std::vector<int> ast, bst;
        for (int D = 0; D <= dmax; ++D) {
            ast.push_back((int)aij.size());
            for (int a = 0; a < M; ++a)
                for (int b = 0; b < M; ++b)
                    if (cfg->lm[2 * a + 1] - cfg->lm[2 * b + 1] == D)
                        aij.push_back((uint16_t)(a | (b << 8)));
        }
        ast.push_back((int)aij.size());
        for (int S = -dmax; S <= dmax; ++S) {
            bst.push_back((int)bij.size());
            for (int a = 0; a < M; ++a)
                for (int b = a; b < M; ++b)
                    if (cfg->lm[2 * a + 1] + cfg->lm[2 * b + 1] == S)
                        bij.push_back((uint16_t)(a | (b << 8)));
        }
        bst.push_back((int)bij.size());
        const int nA = (int)aij.size(), nB = (int)bij.size();
        if ((rc = dalloc(h, &h->aux_q, (size_t)N)) || (rc = dalloc(h, &h->aux_m, (size_t)N)) ||
            (rc = dalloc(h, &h->aux_j, (size_t)N)) || (rc = dalloc(h, &h->fix_idx, (size_t)N)) ||
            (rc = dalloc(h, &h->fix_count, (size_t)4)) || (rc = dalloc(h, &h->fix_aij, (size_t)nA)) ||
            (rc = dalloc(h, &h->fix_bij, (size_t)nB)) || (rc = dalloc(h, &h->fix_astart, ast.size())) ||
            (rc = dalloc(h, &h->fix_bstart, bst.size())) || (rc = dalloc(h, &h->fix_ua, (size_t)K * nA)) ||
            (rc = dalloc(h, &h->fix_vb, (size_t)K * nB)) || (rc = dalloc(h, &h->fix_qdf, (size_t)K * M * cfg->n_q))) {
            release(h);
            return rc;
        }
        if (cudaMemcpyAsync(h->fix_aij, aij.data(), sizeof(uint16_t) * nA, cudaMemcpyHostToDevice, h->stream) ||
            cudaMemcpyAsync(h->fix_bij, bij.data(), sizeof(uint16_t) * nB, cudaMemcpyHostToDevice, h->stream) ||
            cudaMemcpyAsync(h->fix_astart, ast.data(), sizeof(int) * ast.size(), cudaMemcpyHostToDevice, h->stream) ||
            cudaMemcpyAsync(h->fix_bstart, bst.data(), sizeof(int) * bst.size(), cudaMemcpyHostToDevice, h->stream) ||
            cudaStreamSynchronize(h->stream)) {
            cudaGetLastError();
            release(h);
            return RIFT_ECUDA;
        }
        h->fix = FixTables{h->fix_aij, h->fix_astart, h->fix_bij, h->fix_bstart, h->fix_ua, h->fix_vb, h->fix_qdf,
                           nA, nB, dmax};
        // samples with quad32 + |max lin32| above this are corrected: below it the float32
        // rounding stays under 5e-4 (measured, ~3e-7 per unit of the terms at most)
        h->fix_thr = kFixThreshold;
        if (const char *env = std::getenv("RIFT_ILE_FIX_T"))
            h->fix_thr = (float)std::atof(env);
    }
    if (cfg->precision == RIFT_MIXED) {
        h->refine_rows = std::min<int64_t>(N, kRefineRows);
        if ((rc = dalloc(h, &h->refine_bins, (size_t)h->refine_rows * cfg->n_t))) {
            release(h);
            return rc;
        }
    }
    h->host_out.assign(8 + 8 * (RIFT_MAX_ITER + 1) + 8, 0.0);

    // time-bin split table: j * beta = bin_i + bin_f
    std::vector<int> bi(cfg->n_t);
    std::vector<float> bf(cfg->n_t);
    for (int j = 0; j < cfg->n_t; ++j) {
        double jb = (cfg->n_t > 1 ? j * (cfg->t_hi_s - cfg->t_lo_s) / (cfg->n_t - 1) : 0.0) * cfg->fs_hz;
        double fl = std::floor(jb);
        bi[j] = (int)fl;
        bf[j] = (float)(jb - fl);
        if (bf[j] >= 1.0f)
            bf[j] = 0x1.fffffep-1f;
    }
    std::vector<double> P0((size_t)6 * B, 1.0 / B);
    if (cudaMemcpyAsync(h->bin_i, bi.data(), sizeof(int) * cfg->n_t, cudaMemcpyHostToDevice, h->stream) ||
        cudaMemcpyAsync(h->bin_f, bf.data(), sizeof(float) * cfg->n_t, cudaMemcpyHostToDevice, h->stream) ||
        cudaMemcpyAsync(h->P, P0.data(), sizeof(double) * 6 * B, cudaMemcpyHostToDevice, h->stream) ||
        cudaMemsetAsync(h->err, 0, sizeof(int) * 4, h->stream) ||
        cudaMemsetAsync(h->iter_dev, 0, sizeof(uint32_t) * 4, h->stream) || launch_build_cdf(sampler_of(h), h->stream) ||
        cudaStreamSynchronize(h->stream)) {
        cudaGetLastError();
        release(h);
        return RIFT_ECUDA;
    }
    P.tc_groups = (cfg->n_q + 7) / 8 + 17;
    P.Qtc = h->Qtc;
    P.qmax_bits = h->qmax_bits;
    {
        int dev = 0, max_smem = 0, major = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        h->tc_ok = major == 10 && lnl_tc_fits(P, max_smem);
        const char *env = std::getenv("RIFT_ILE_TC");
        if (env && env[0] == '0')
            h->tc_mode = 0;
        else if (env && env[0] == '1')
            h->tc_mode = 1;
        if (prepare_sampler_kernels() != cudaSuccess || prepare_refine_kernels() != cudaSuccess ||
            prepare_tile_kernels() != cudaSuccess || (h->tc_ok && prepare_tc_kernels() != cudaSuccess) ||
            prepare_fix_kernels() != cudaSuccess) {
            cudaGetLastError();
            release(h);
            return RIFT_ECUDA;
        }
    }
    P.Q64 = h->Q64;
    P.U64 = h->U64;
    P.V64 = h->V64;
    P.Qr32 = h->Qr32;
    P.U32 = h->U32;
    P.V32 = h->V32;
    P.Ttc = h->Ttc;
    P.tt_exp = h->tt_exp;
    *out = h;
    return RIFT_OK;
}

void rift_ile_destroy(rift_ile_t *h) { release(h); }

int64_t rift_ile_kernel_launches(const rift_ile_t *h) { return h ? h->launches : -1; }

int rift_ile_get_plan(const rift_ile_t *h, int32_t *lnl_kernel, int32_t *samples_per_cell)
{
    if (!h)
        return RIFT_EINVAL;
    const int64_t n = h->last_n > 0 ? h->last_n : h->cap;
    if (lnl_kernel)
        *lnl_kernel = !use_fp32(h) ? RIFT_KERNEL_FP64 : use_tc(h, n) ? RIFT_KERNEL_TENSOR : RIFT_KERNEL_CUDA_CORE;
    if (samples_per_cell)
        *samples_per_cell = h->plan.per_cell;
    return RIFT_OK;
}

int64_t rift_ile_footprint(const rift_ile_config *cfg)
{
    if (validate(cfg) != RIFT_OK)
        return -1;
    const int64_t K = cfg->n_det, M = cfg->n_modes, N = cfg->max_samples, B = cfg->n_bins, nt = cfg->n_t;
    const int64_t nq = cfg->n_q, nq_pad = ((nq + 3) & ~3) + kQPad;
    const int64_t groups = (nq + 7) / 8 + 17, kp = (2 * M + 15) / 16 * 16;
    const int64_t sizes[] = {
        K * M * nq * 16, 2 * K * M * M * 16, K * 2 * M * nq_pad * 4, 2 * K * M * M * 8, K * 2 * kp * kp * 2, K * 4,
        2 * nt * 4,
        N * 6 * 8, 3 * N * 8, N * 8, 2 * N * 4, (int64_t)sort_scratch_words(N) * 4, 16, 16,
        K * 2 * groups * kp * 8 * 2, 5 * kRedBlocks * 8, 152 * 12 * B * 8, 8 * (RIFT_MAX_ITER + 1) * 8, 3 * 8 * 8,
        N * 4, 16, 6 * B * 8, 6 * (B + 1) * 8, 6 * B * 8, 16, (int64_t)kSelectWords * 4,
        cfg->precision == RIFT_MIXED ? std::min<int64_t>(N, kRefineRows) * nt * 8 : 0,
        // large-term correction: per-sample side outputs and list, pair tables, double-float
        // copies of U, V (at most M^2 pairs each) and Q
        cfg->precision != RIFT_FP64 && !cfg->distance_marg ? 4 * N * 4 + 16 + 4 * M * M + 8 * 64 +
                                                                  2 * K * M * M * 16 + K * M * nq * 16
                                                            : 0};
    int64_t total = 0;
    for (int64_t b : sizes)
        total += b + 16;
    return total + 64 * 1024;   // event and stream bookkeeping slack
}

int rift_ile_set_overlaps(rift_ile_t *h, const void *Q, const void *U, const void *V, int mem)
{
    if (!h || !Q || !U || !V || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE))
        return RIFT_EINVAL;
    const int K = h->prob.K, M = h->prob.M, nq = h->prob.n_q;
    const size_t qb = sizeof(double2) * (size_t)K * M * nq, gb = sizeof(double2) * (size_t)K * M * M;
    const cudaMemcpyKind kind = mem == RIFT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // symmetry checks on host copies of U, V (Sec. V A: U^* = U^T, V = V^T)
    std::vector<double> hu(2 * (size_t)K * M * M), hv(2 * (size_t)K * M * M);
    if (mem == RIFT_MEM_HOST) {
        std::memcpy(hu.data(), U, gb);
        std::memcpy(hv.data(), V, gb);
    } else {
        CK(cudaMemcpyAsync(hu.data(), U, gb, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(hv.data(), V, gb, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    for (int k = 0; k < K; ++k) {
        double su = 0, sv = 0;
        for (size_t e = 0; e < (size_t)2 * M * M; ++e) {
            double a = std::fabs(hu[2 * (size_t)k * M * M + e]), b = std::fabs(hv[2 * (size_t)k * M * M + e]);
            if (!std::isfinite(a) || !std::isfinite(b))
                return RIFT_ENONFINITE;
            su = std::max(su, a);
            sv = std::max(sv, b);
        }
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) {
                size_t ab = 2 * (((size_t)k * M + a) * M + b), ba = 2 * (((size_t)k * M + b) * M + a);
                if (std::fabs(hu[ab] - hu[ba]) > 1e-10 * su || std::fabs(hu[ab + 1] + hu[ba + 1]) > 1e-10 * su)
                    return RIFT_EINVAL;
                if (std::fabs(hv[ab] - hv[ba]) > 1e-10 * sv || std::fabs(hv[ab + 1] - hv[ba + 1]) > 1e-10 * sv)
                    return RIFT_EINVAL;
            }
    }
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    CK(cudaMemcpyAsync(h->Q64, Q, qb, kind, h->stream));
    CK(cudaMemcpyAsync(h->U64, U, gb, kind, h->stream));
    CK(cudaMemcpyAsync(h->V64, V, gb, kind, h->stream));
    return install_overlaps(h);
}

int rift_ile_set_waveforms(rift_ile_t *h, int32_t n_freq, const double *freqs, const void *hlm, const void *data,
                           const double *weights, int mem)
{
    if (!h || n_freq < 2 || !freqs || !hlm || !data || !weights || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE))
        return RIFT_EINVAL;
    const int K = h->prob.K, M = h->prob.M, F = n_freq;
    const size_t fb = sizeof(double) * F, hb = sizeof(double2) * (size_t)M * F, db = sizeof(double2) * (size_t)K * F,
                 wb = sizeof(double) * (size_t)K * F;
    // host checks: mirror-symmetric grid, weights finite, non-negative and symmetric in f
    std::vector<double> hf(F), hw((size_t)K * F);
    const cudaMemcpyKind to_host = mem == RIFT_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(hf.data(), freqs, fb, to_host, h->stream));
    CK(cudaMemcpyAsync(hw.data(), weights, wb, to_host, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < F; ++j) {
        if (!std::isfinite(hf[j]) || hf[F - 1 - j] != -hf[j])
            return RIFT_EINVAL;
        for (int k = 0; k < K; ++k) {
            const double a = hw[(size_t)k * F + j];
            if (!std::isfinite(a))
                return RIFT_ENONFINITE;
            if (a < 0.0 || a != hw[(size_t)k * F + (F - 1 - j)])
                return RIFT_EINVAL;
        }
    }
    std::vector<void *> tmp;
    auto grab = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMallocAsync(&q, bytes, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        tmp.push_back(q);
        return q;
    };
    auto A = static_cast<double2 *>(grab(sizeof(double2) * (size_t)K * M * F));
    auto t0 = static_cast<double *>(grab(sizeof(double) * K));
    // Q by FFT when the grid lies on a lattice f_j = f_0 + n_j df (ascending, integer n_j
    // within 1e-9 relative) and L = f_s / df is a power of two spanning every n_j; else the
    // direct sum.  RIFT_ILE_DFT=1 forces the direct sum.
    FftPlan plan{};
    bool use_fft = !(std::getenv("RIFT_ILE_DFT") && std::getenv("RIFT_ILE_DFT")[0] == '1');
    std::vector<int> nidx(F);
    {
        double df = 0.0, fmax = 0.0;
        for (int j = 0; j < F; ++j)
            fmax = std::max(fmax, std::fabs(hf[j]));
        for (int j = 1; j < F && use_fft; ++j) {
            const double gap = hf[j] - hf[j - 1];
            if (!(gap > 0.0))
                use_fft = false;
            else if (df == 0.0 || gap < df)
                df = gap;
        }
        const double Lr = use_fft && df > 0.0 ? h->prob.fs / df : 0.0;
        const int64_t L = (int64_t)std::llround(Lr);
        use_fft = use_fft && L >= 2 && L <= ((int64_t)1 << 26) && (L & (L - 1)) == 0 &&
                  std::fabs(Lr - (double)L) <= 1e-9 * (double)L;
        for (int j = 0; j < F && use_fft; ++j) {
            const double nr = (hf[j] - hf[0]) / df;
            const int64_t nj = std::llround(nr);
            if (std::fabs(hf[j] - hf[0] - (double)nj * df) > 1e-9 * std::max(1.0, fmax) || nj < 0 || nj >= L)
                use_fft = false;
            else
                nidx[j] = (int)nj;
        }
        if (use_fft) {
            plan.L = (int)L;
            plan.f0 = hf[0];
            auto ni = static_cast<int *>(grab(sizeof(int) * F));
            plan.X = static_cast<double2 *>(grab(sizeof(double2) * (size_t)K * M * L));
            plan.Y = static_cast<double2 *>(grab(sizeof(double2) * (size_t)K * M * L));
            plan.T = static_cast<double2 *>(grab(sizeof(double2) * (size_t)std::max<int64_t>(1, L / 2)));
            if (!ni || !plan.X || !plan.Y || !plan.T ||
                cudaMemcpyAsync(ni, nidx.data(), sizeof(int) * F, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                use_fft = false;   // the direct sum needs no scratch of this size
            plan.nidx = ni;
        }
    }
    int launched = 0;
    const double *df = freqs, *dw = weights;
    const double2 *dh = static_cast<const double2 *>(hlm), *dd = static_cast<const double2 *>(data);
    int rc = (A && t0) ? RIFT_OK : RIFT_ENOMEM;
    if (rc == RIFT_OK && mem == RIFT_MEM_HOST) {
        auto f2 = static_cast<double *>(grab(fb));
        auto h2 = static_cast<double2 *>(grab(hb));
        auto d2 = static_cast<double2 *>(grab(db));
        auto w2 = static_cast<double *>(grab(wb));
        if (!f2 || !h2 || !d2 || !w2)
            rc = RIFT_ENOMEM;
        else if (cudaMemcpyAsync(f2, freqs, fb, cudaMemcpyHostToDevice, h->stream) ||
                 cudaMemcpyAsync(h2, hlm, hb, cudaMemcpyHostToDevice, h->stream) ||
                 cudaMemcpyAsync(d2, data, db, cudaMemcpyHostToDevice, h->stream) ||
                 cudaMemcpyAsync(w2, weights, wb, cudaMemcpyHostToDevice, h->stream))
            rc = RIFT_ECUDA;
        df = f2;
        dh = h2;
        dd = d2;
        dw = w2;
    }
    if (rc == RIFT_OK &&
        (cudaMemcpyAsync(t0, h->q_t0.data(), sizeof(double) * K, cudaMemcpyHostToDevice, h->stream) ||
         cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) ||
         launch_precompute(dh, dd, dw, df, K, M, F, t0, h->prob.fs, h->prob.n_q, A, h->Q64, h->U64, h->V64,
                           h->stream, use_fft ? &plan : nullptr, &launched)))
        rc = RIFT_ECUDA;
    if (rc == RIFT_OK)
        h->launches += launched;
    for (void *q : tmp)
        cudaFreeAsync(q, h->stream);
    if (rc != RIFT_OK) {
        cudaStreamSynchronize(h->stream);
        cudaGetLastError();
        return rc;
    }
    return install_overlaps(h);
}

}  // extern "C"

namespace rift {
namespace host {

// float32 and tensor-core copies of the overlaps now in Q64/U64/V64; marks them set.
int install_overlaps(rift_ile_t *h)
{
    const int K = h->prob.K, M = h->prob.M, nq = h->prob.n_q;
    int64_t tot = (int64_t)K * 2 * M * h->prob.n_q_pad;
    int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 8);
    prep_overlaps_kernel<<<grid, 256, 0, h->stream>>>(h->Q64, h->U64, h->V64, K, M, nq, h->prob.n_q_pad, h->Qr32,
                                                      h->U32, h->V32, h->err);
    CK(cudaGetLastError());
    h->launches += 1;
    if (h->tc_ok) {
        CK(launch_prep_tc(h->Q64, K, M, nq, h->prob.tc_groups, h->qmax_bits, h->Qtc, h->stream));
        CK(launch_prep_tt(h->U64, h->V64, K, M, h->Ttc, h->tt_exp, h->stream));
        h->launches += 3;
    }
    if (h->fix_on) {
        CK(launch_fix_prep(h->prob, h->fix, h->fix_ua, h->fix_vb, h->fix_qdf, h->stream));
        h->launches += 1;
    }
    int rc = sync_and_err(h);
    h->have_overlaps = (rc == RIFT_OK);
    return rc;
}

}  // namespace host
}  // namespace rift

extern "C" {

int rift_ile_wait_selftest(rift_ile_t *h, int64_t limit_ns)
{
    if (!h || limit_ns < 1000 || limit_ns > 2000000000)
        return RIFT_EINVAL;
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    CK(launch_wait_probe((uint64_t)limit_ns, h->err, h->stream));
    h->launches += 1;
    return sync_and_err(h);
}

int rift_ile_get_overlaps(const rift_ile_t *h, void *Q, void *U, void *V, int mem)
{
    if (!h || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE))
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    const int K = h->prob.K, M = h->prob.M;
    const cudaMemcpyKind kind = mem == RIFT_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (Q)
        CK(cudaMemcpyAsync(Q, h->Q64, sizeof(double2) * (size_t)K * M * h->prob.n_q, kind, h->stream));
    if (U)
        CK(cudaMemcpyAsync(U, h->U64, sizeof(double2) * (size_t)K * M * M, kind, h->stream));
    if (V)
        CK(cudaMemcpyAsync(V, h->V64, sizeof(double2) * (size_t)K * M * M, kind, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RIFT_OK;
}

int rift_ile_eval(rift_ile_t *h, const double *theta, int64_t n, int mem, double *lnL_tmarg, double *lnL_t)
{
    if (!h || n < 0 || (n > 0 && (!theta || !lnL_tmarg)) || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE))
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    if (n == 0)
        return RIFT_OK;
    const int nt = h->prob.n_t;
    int64_t chunk = h->cap;
    double *stage_t = nullptr;
    if (lnL_t && mem == RIFT_MEM_HOST) {
        chunk = std::min<int64_t>(chunk, std::max<int64_t>(1, (int64_t)(64 << 20) / nt));
        void *q = nullptr;
        if (cudaMallocAsync(&q, sizeof(double) * (size_t)chunk * nt, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return RIFT_ENOMEM;
        }
        stage_t = static_cast<double *>(q);
    }
    int rc = RIFT_OK;
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    h->last_n = 0;   // the staging buffers no longer hold a drawn batch
    for (int64_t i0 = 0; i0 < n && rc == RIFT_OK; i0 += chunk) {
        const int64_t c = std::min(chunk, n - i0);
        const double *th = theta + 6 * i0;
        double *o = lnL_tmarg + i0;
        double *ot = lnL_t ? lnL_t + i0 * nt : nullptr;
        if (mem == RIFT_MEM_HOST) {
            if (cudaMemcpyAsync(h->theta, th, sizeof(double) * 6 * c, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
                rc = RIFT_ECUDA;
                break;
            }
            rc = eval_device(h, h->theta, c, h->lnL, stage_t, nullptr, nullptr);
            if (rc == RIFT_OK &&
                (cudaMemcpyAsync(o, h->lnL, sizeof(double) * c, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
                 (ot && cudaMemcpyAsync(ot, stage_t, sizeof(double) * c * nt, cudaMemcpyDeviceToHost, h->stream) !=
                            cudaSuccess)))
                rc = RIFT_ECUDA;
        } else {
            rc = eval_device(h, th, c, o, ot, nullptr, nullptr);
        }
    }
    if (stage_t)
        cudaFreeAsync(stage_t, h->stream);
    int rc2 = sync_and_err(h);
    return rc != RIFT_OK ? rc : rc2;
}

int rift_ile_coeffs(rift_ile_t *h, const double *theta, int64_t n, int mem, double *c, double *dt, double *quad)
{
    if (!h || n < 0 || (n > 0 && !theta) || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE))
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    if (n == 0)
        return RIFT_OK;
    const bool fp64 = h->cfg.precision == RIFT_FP64;
    const int K = h->prob.K, M = h->prob.M;
    if (mem == RIFT_MEM_DEVICE) {
        CK(launch_coeffs(h->prob, fp64, theta, n, reinterpret_cast<double2 *>(c), dt, quad, h->stream));
        return sync_and_err(h);
    }
    const int64_t chunk = std::min<int64_t>(h->cap, 1 << 16);
    double2 *dc = nullptr;
    double *ddt = nullptr, *dq = nullptr;
    std::vector<void *> tmp;
    auto grab = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMallocAsync(&q, bytes, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        tmp.push_back(q);
        return q;
    };
    dc = static_cast<double2 *>(grab(sizeof(double2) * chunk * K * M));
    ddt = static_cast<double *>(grab(sizeof(double) * chunk * K));
    dq = static_cast<double *>(grab(sizeof(double) * chunk));
    int rc = (dc && ddt && dq) ? RIFT_OK : RIFT_ENOMEM;
    for (int64_t i0 = 0; i0 < n && rc == RIFT_OK; i0 += chunk) {
        const int64_t m = std::min(chunk, n - i0);
        if (cudaMemcpyAsync(h->theta, theta + 6 * i0, sizeof(double) * 6 * m, cudaMemcpyHostToDevice, h->stream) ||
            launch_coeffs(h->prob, fp64, h->theta, m, c ? dc : nullptr, dt ? ddt : nullptr, quad ? dq : nullptr,
                          h->stream) ||
            (c && cudaMemcpyAsync(c + 2 * i0 * K * M, dc, sizeof(double2) * m * K * M, cudaMemcpyDeviceToHost,
                                  h->stream)) ||
            (dt && cudaMemcpyAsync(dt + i0 * K, ddt, sizeof(double) * m * K, cudaMemcpyDeviceToHost, h->stream)) ||
            (quad && cudaMemcpyAsync(quad + i0, dq, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream)))
            rc = RIFT_ECUDA;
    }
    for (void *q : tmp)
        cudaFreeAsync(q, h->stream);
    cudaStreamSynchronize(h->stream);
    h->last_n = 0;
    cudaGetLastError();
    return rc;
}

int rift_ile_marginalize(rift_ile_t *h, int64_t n_samples, rift_ile_result *out)
{
    if (!h || n_samples < 1 || n_samples > h->cap)
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    RK(choose_plan(h, n_samples));
    RK(ensure_events(h, 1));
    h->timed = true;
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    RK(run_iteration(h, n_samples, 0, false, true));
    CK(launch_pooled_final(h->pooled, h->final_out, h->iter_dev, 1, h->stream));
    h->launches += 1;
    h->iteration += 1;
    h->last_n = n_samples;
    return collect_result(h, 1, out);
}

int rift_ile_adapt(rift_ile_t *h, int32_t n_iter, int64_t n_per_iter, rift_ile_result *out)
{
    if (!h || n_iter < 1 || n_iter > RIFT_MAX_ITER || n_per_iter < 1 || n_per_iter > h->cap)
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    RK(choose_plan(h, n_per_iter));
    RK(ensure_events(h, n_iter));
    h->timed = true;
    const bool same_graph = h->graph && h->graph_iter == n_iter && h->graph_n == n_per_iter &&
                            h->graph_plan == h->plan;
    const bool repeat = h->last_shape_iter == n_iter && h->last_shape_n == n_per_iter;
    if (graphs_enabled() && (same_graph || repeat)) {
        // a repeated shape: capture once, then replay
        if (!same_graph)
            RK(capture_adapt(h, n_iter, n_per_iter));
        CK(cudaGraphLaunch(h->graph, h->stream));
        h->launches += h->graph_launches;
    } else {
        RK(enqueue_adapt(h, n_iter, n_per_iter));
    }
    h->last_shape_iter = n_iter;
    h->last_shape_n = n_per_iter;
    h->iteration += (uint32_t)n_iter;
    h->last_n = n_per_iter;
    return collect_result(h, n_iter, out);
}

int rift_ile_last_batch(rift_ile_t *h, int mem, double *theta, double *lnp_minus_lnps, double *lnL_tmarg, double *lnw,
                        int64_t *n_out)
{
    if (!h || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE))
        return RIFT_EINVAL;
    const int64_t n = h->last_n;
    if (n_out)
        *n_out = n;
    if (n == 0)
        return RIFT_ESTATE;
    const cudaMemcpyKind kind = mem == RIFT_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (theta)
        CK(cudaMemcpyAsync(theta, h->theta, sizeof(double) * 6 * n, kind, h->stream));
    if (lnp_minus_lnps)
        CK(cudaMemcpyAsync(lnp_minus_lnps, h->lnpw, sizeof(double) * n, kind, h->stream));
    if (lnL_tmarg)
        CK(cudaMemcpyAsync(lnL_tmarg, h->lnL, sizeof(double) * n, kind, h->stream));
    if (lnw)
        CK(cudaMemcpyAsync(lnw, h->lnw, sizeof(double) * n, kind, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RIFT_OK;
}

int rift_ile_fair_draws(rift_ile_t *h, int64_t n_draws, uint64_t seed, int mem, double *theta, double *t,
                        int64_t *index)
{
    if (!h || n_draws < 0 || (mem != RIFT_MEM_HOST && mem != RIFT_MEM_DEVICE) || h->cfg.distance_marg)
        return RIFT_EINVAL;
    if (n_draws == 0)
        return RIFT_OK;
    if (!theta && !t && !index)
        return RIFT_EINVAL;
    const int64_t n = h->last_n;
    if (n == 0)
        return RIFT_ESTATE;
    const int nt = h->prob.n_t;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_draws, (int64_t)(16 << 20) / nt));
    std::vector<void *> tmp;
    auto grab = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMallocAsync(&q, bytes, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        tmp.push_back(q);
        return q;
    };
    auto W = static_cast<uint64_t *>(grab(sizeof(uint64_t) * n));
    auto E = static_cast<uint64_t *>(grab(sizeof(uint64_t) * n));
    auto scan = static_cast<uint64_t *>(grab(sizeof(uint64_t) * scan_scratch_words(n)));
    auto idx = static_cast<int64_t *>(grab(sizeof(int64_t) * n_draws));
    auto th = static_cast<double *>(grab(sizeof(double) * 6 * n_draws));
    auto Ut = static_cast<uint64_t *>(grab(sizeof(uint64_t) * n_draws));
    auto tt = static_cast<double *>(grab(sizeof(double) * n_draws));
    auto jj = static_cast<int32_t *>(grab(sizeof(int32_t) * n_draws));
    auto bins = static_cast<double *>(grab(sizeof(double) * chunk * nt));
    auto lt = static_cast<double *>(grab(sizeof(double) * chunk));
    int rc = (W && E && scan && idx && th && Ut && tt && jj && bins && lt) ? RIFT_OK : RIFT_ENOMEM;
    const cudaMemcpyKind kind = mem == RIFT_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    auto run = [&]() -> int {
        CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
        // the batch's largest ln w (checks every ln w is finite)
        CK(launch_reduce(h->lnw, h->lnL, n, h->red_partial, h->stats, kScratchSlot, h->pooled_scratch, 1, h->err,
                         h->stream));
        int k = 0;
        CK(launch_fair_select(h->lnw, n, h->stats, kScratchSlot, W, E, scan, seed, n_draws, h->theta, idx, th, Ut,
                              h->stream, &k));
        h->launches += 2 + k;
        // time bins from each drawn sample's per-bin ln L, in float64 (the draws are few)
        for (int64_t c0 = 0; c0 < n_draws; c0 += chunk) {
            const int64_t m = std::min(chunk, n_draws - c0);
            CK(launch_lnl_fp64(h->prob, th + 6 * c0, m, lt, bins, nullptr, nullptr, h->err, h->stream));
            CK(launch_fair_time(bins, m, nt, Ut + c0, h->prob.t_lo, h->prob.t_step, jj + c0, tt + c0, h->stream));
            h->launches += 2;
        }
        if (theta)
            CK(cudaMemcpyAsync(theta, th, sizeof(double) * 6 * n_draws, kind, h->stream));
        if (t)
            CK(cudaMemcpyAsync(t, tt, sizeof(double) * n_draws, kind, h->stream));
        if (index)
            CK(cudaMemcpyAsync(index, idx, sizeof(int64_t) * n_draws, kind, h->stream));
        return RIFT_OK;
    };
    if (rc == RIFT_OK)
        rc = run();
    for (void *q : tmp)
        cudaFreeAsync(q, h->stream);
    const int rc2 = sync_and_err(h);
    return rc != RIFT_OK ? rc : rc2;
}

int rift_ile_get_sampler(const rift_ile_t *h, double *P)
{
    if (!h || !P)
        return RIFT_EINVAL;
    CK(cudaMemcpyAsync(P, h->P, sizeof(double) * 6 * h->cfg.n_bins, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RIFT_OK;
}

int rift_ile_get_state(const rift_ile_t *h, void *buf, size_t *len)
{
    if (!h || !len)
        return RIFT_EINVAL;
    const size_t need = sizeof(StateHeader) + sizeof(double) * 6 * h->cfg.n_bins;
    if (!buf) {
        *len = need;
        return RIFT_OK;
    }
    if (*len < need)
        return RIFT_EINVAL;
    StateHeader hd{kStateMagic, kStateVersion, (uint32_t)h->cfg.n_bins, h->cfg.seed, h->iteration, 0};
    std::memcpy(buf, &hd, sizeof(hd));
    int rc = rift_ile_get_sampler(h, reinterpret_cast<double *>(static_cast<char *>(buf) + sizeof(hd)));
    if (rc != RIFT_OK)
        return rc;
    *len = need;
    return RIFT_OK;
}

int rift_ile_set_state(rift_ile_t *h, const void *buf, size_t len)
{
    if (!h || !buf)
        return RIFT_EINVAL;
    const size_t need = sizeof(StateHeader) + sizeof(double) * 6 * h->cfg.n_bins;
    if (len != need)
        return RIFT_ESTATE;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.n_bins != (uint32_t)h->cfg.n_bins)
        return RIFT_ESTATE;
    const double *P = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof(hd));
    for (int e = 0; e < 6 * h->cfg.n_bins; ++e)
        if (!(P[e] >= 0.0) || !std::isfinite(P[e]))
            return RIFT_ESTATE;
    drop_graph(h);   // the seed is a kernel argument of the captured draws
    h->cfg.seed = hd.seed;
    h->iteration = hd.iteration;
    CK(cudaMemcpyAsync(h->iter_dev, &h->iteration, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->P, P, sizeof(double) * 6 * h->cfg.n_bins, cudaMemcpyHostToDevice, h->stream));
    CK(launch_build_cdf(sampler_of(h), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->last_n = 0;
    return RIFT_OK;
}

}  // extern "C"
