// Sampler, sort and reduction kernels of the ILE hot path.
//
//   draw      - product-form adaptive sampling prior (arXiv:2505.11655 Sec. II B): every
//               extrinsic coordinate is drawn through its prior-CDF coordinate v in [0,1)
//               from a B-bin histogram, so p/p_s = prod_d 1 / (B P_d[b_d] / sum_b P_d[b]).
//   sort      - counting sort of samples by sky cell (keeps a tile's Q windows close).
//   reduce    - ln Z = ln mean w, sigma, n_eff = sum w / max w (Eq. (neff)),
//               n_ESS = (sum w)^2 / sum w^2 (Sec. IV A), all in float64, deterministic
//               two-level reductions.
//   adapt     - 1-D weighted histograms of the weights, mixed with a uniform floor.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>

#include "ile_kernels.h"

namespace rift {

// ======================================================================== draw

constexpr int kDrawThreads = 256;

__global__ void __launch_bounds__(kDrawThreads) draw_kernel(SamplerDev S, SkyGrid G, uint32_t iter, int64_t n,
                                                            double *__restrict__ theta, double *__restrict__ lnpw,
                                                            uint64_t *__restrict__ bins, uint32_t *__restrict__ key)
{
    extern __shared__ double sC[];   // [6][B+1] running sums, then [6][B] masses, [6][B] log densities
    const int B = S.B;
    double *sP = sC + 6 * (B + 1);
    double *sL = sP + 6 * B;
    for (int e = threadIdx.x; e < 6 * (B + 1); e += blockDim.x)
        sC[e] = S.C[e];
    for (int e = threadIdx.x; e < 6 * B; e += blockDim.x) {
        sP[e] = S.P[e];
        sL[e] = S.L[e];
    }
    __syncthreads();
    const uint32_t k0 = (uint32_t)S.seed, k1 = (uint32_t)(S.seed >> 32);
    const double d3lo = S.d_min * S.d_min * S.d_min, d3hi = S.d_max * S.d_max * S.d_max;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double u[6];
#pragma unroll
        for (uint32_t p = 0; p < 3; ++p) {
            U4 r = philox10(U4{(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), iter, p}, k0, k1);
            u[2 * p] = unit53(r.x, r.y);
            u[2 * p + 1] = unit53(r.z, r.w);
        }
        double v[6], lr = 0.0;
        uint64_t packed = 0;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const double *Cd = sC + d * (B + 1);
            const double tot = Cd[B];
            const double x = u[d] * tot;
            // last b in [0, B-1] with C[b] <= x (C[0] = 0 <= x always)
            int lo = 0, hi = B - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (Cd[mid] <= x)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const double pb = sP[d * B + lo];
            double t = (x - Cd[lo]) / pb;
            if (!(t >= 0.0))
                t = 0.0;
            if (t >= 1.0)
                t = 0x1.fffffffffffffp-1;
            v[d] = (lo + t) / B;
            lr -= sL[d * B + lo];   // ln(B pb / tot), tabulated when the masses change
            packed |= (uint64_t)lo << (10 * d);
        }
        double th[6];
        th[0] = 2.0 * kPi * v[0];
        th[1] = asin(2.0 * v[1] - 1.0);
        th[2] = kPi * v[2];
        th[3] = 2.0 * kPi * v[3];
        th[4] = acos(1.0 - 2.0 * v[4]);
        th[5] = cbrt(d3lo + v[5] * (d3hi - d3lo));
        double *out = theta + 6 * i;
#pragma unroll
        for (int d = 0; d < 6; ++d)
            out[d] = th[d];
        lnpw[i] = lr;
        bins[i] = packed;
        key[i] = sky_cell(th[0], th[1], G);
    }
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static int grid_for(int64_t n, int threads, int per_sm)
{
    int64_t want = (n + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_draw(const SamplerDev &S, const SkyGrid &G, uint32_t iter, int64_t n, double *theta, double *lnpw,
                        uint64_t *bins, uint32_t *key, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    size_t smem = sizeof(double) * (6 * (S.B + 1) + 12 * S.B);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem(draw_kernel);
        if (e != cudaSuccess)
            return e;
    }
    draw_kernel<<<grid_for(n, kDrawThreads, 8), kDrawThreads, smem, st>>>(S, G, iter, n, theta, lnpw, bins, key);
    return cudaGetLastError();
}

__global__ void keys_kernel(SkyGrid G, const double *__restrict__ theta, int64_t n, uint32_t *__restrict__ key)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = sky_cell(theta[6 * i], theta[6 * i + 1], G);
}

cudaError_t launch_keys(const SkyGrid &G, const double *theta, int64_t n, uint32_t *key, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    keys_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(G, theta, n, key);
    return cudaGetLastError();
}

SkyGrid sky_grid_for(int64_t n)
{
    int order = 4;   // about four samples per cell
    while (order < kMaxOrder && ((int64_t)4 << (2 * order)) < n)
        ++order;
    return SkyGrid{order, 1 << (2 * order)};
}

// ======================================================================== counting sort by sky cell

__global__ void count_kernel(const uint32_t *__restrict__ key, int64_t n, uint32_t *__restrict__ counts)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + key[i], 1u);
}

// Exclusive scan of the n_cells counts in three passes: per-block totals of 4096
// counts, a scan of those totals by one block, then a block-level scan of each
// 4096-count slice offset by its total.  Loads and stores are coalesced; each
// thread owns 16 consecutive counts staged through shared memory.
constexpr int kScanTile = 4096;
constexpr int kScanThreads = 256;

__global__ void __launch_bounds__(kScanThreads) scan_totals_kernel(const uint32_t *__restrict__ counts, int n_cells,
                                                                   uint32_t *__restrict__ totals)
{
    __shared__ uint32_t red[kScanThreads / 32];
    const int base = blockIdx.x * kScanTile;
    uint32_t v = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        if (base + i < n_cells)
            v += counts[base + i];
#pragma unroll
    for (int o = 16; o; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w)
            t += red[w];
        totals[blockIdx.x] = t;
    }
}

// Block-wide exclusive scan of one value per thread; returns this thread's offset.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return x - v + (w > 0 ? warp_tot[w - 1] : 0u);
}

__global__ void __launch_bounds__(1024) scan_top_kernel(uint32_t *totals, int nb)
{
    __shared__ uint32_t warp_tot[32];
    const uint32_t v = threadIdx.x < nb ? totals[threadIdx.x] : 0u;
    const uint32_t e = block_exclusive_scan(v, warp_tot);
    if (threadIdx.x < nb)
        totals[threadIdx.x] = e;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(uint32_t *__restrict__ counts, int n_cells,
                                                                  const uint32_t *__restrict__ totals)
{
    constexpr int per = kScanTile / kScanThreads;
    __shared__ uint32_t tile[kScanTile + kScanTile / 32];   // padded: thread-strided reads avoid conflicts
    __shared__ uint32_t warp_tot[32];
    const int base = blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        tile[i + (i >> 5)] = base + i < n_cells ? counts[base + i] : 0u;
    __syncthreads();
    uint32_t loc[per], run = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int i = threadIdx.x * per + q;
        loc[q] = run;
        run += tile[i + (i >> 5)];
    }
    const uint32_t off = block_exclusive_scan(run, warp_tot) + totals[blockIdx.x];
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int i = threadIdx.x * per + q;
        tile[i + (i >> 5)] = off + loc[q];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        if (base + i < n_cells)
            counts[base + i] = tile[i + (i >> 5)];
}

__global__ void scatter_kernel(const uint32_t *__restrict__ key, int64_t n, uint32_t *__restrict__ offs,
                               uint32_t *__restrict__ perm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t pos = atomicAdd(offs + key[i], 1u);
        perm[pos] = (uint32_t)i;
    }
}

cudaError_t launch_sort(const SkyGrid &G, const uint32_t *key, int64_t n, uint32_t *counts, uint32_t *perm,
                        cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (G.n_cells + 1), st);
    if (e != cudaSuccess)
        return e;
    const int g = grid_for(n, 256, 8);
    count_kernel<<<g, 256, 0, st>>>(key, n, counts);
    const int nb = (G.n_cells + kScanTile - 1) / kScanTile;   // <= 256 for 2^20 cells
    uint32_t *totals = counts + kMaxCells + 1;
    scan_totals_kernel<<<nb, kScanThreads, 0, st>>>(counts, G.n_cells, totals);
    scan_top_kernel<<<1, 1024, 0, st>>>(totals, nb);
    scan_apply_kernel<<<nb, kScanThreads, 0, st>>>(counts, G.n_cells, totals);
    scatter_kernel<<<g, 256, 0, st>>>(key, n, counts, perm);
    return cudaGetLastError();
}

// ======================================================================== reductions (float64)

constexpr int kRedThreads = 256;

struct Acc {
    double mx, s1, s2, lmx;
    int bad;
};

__device__ __forceinline__ Acc acc_merge(Acc a, Acc b)
{
    Acc r;
    r.mx = fmax(a.mx, b.mx);
    double fa = (a.mx == -INFINITY) ? 0.0 : exp(a.mx - r.mx);
    double fb = (b.mx == -INFINITY) ? 0.0 : exp(b.mx - r.mx);
    r.s1 = a.s1 * fa + b.s1 * fb;
    r.s2 = a.s2 * fa * fa + b.s2 * fb * fb;
    r.lmx = fmax(a.lmx, b.lmx);
    r.bad = a.bad | b.bad;
    return r;
}

__device__ Acc block_merge(Acc a)
{
    __shared__ double smx[32], ss1[32], ss2[32], slm[32];
    __shared__ int sbad[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        Acc b;
        b.mx = __shfl_xor_sync(0xffffffffu, a.mx, o);
        b.s1 = __shfl_xor_sync(0xffffffffu, a.s1, o);
        b.s2 = __shfl_xor_sync(0xffffffffu, a.s2, o);
        b.lmx = __shfl_xor_sync(0xffffffffu, a.lmx, o);
        b.bad = __shfl_xor_sync(0xffffffffu, a.bad, o);
        a = acc_merge(a, b);
    }
    if (lane == 0) {
        smx[w] = a.mx;
        ss1[w] = a.s1;
        ss2[w] = a.s2;
        slm[w] = a.lmx;
        sbad[w] = a.bad;
    }
    __syncthreads();
    if (w == 0) {
        Acc b = lane < nw ? Acc{smx[lane], ss1[lane], ss2[lane], slm[lane], sbad[lane]}
                          : Acc{-INFINITY, 0.0, 0.0, -INFINITY, 0};
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            Acc c;
            c.mx = __shfl_xor_sync(0xffffffffu, b.mx, o);
            c.s1 = __shfl_xor_sync(0xffffffffu, b.s1, o);
            c.s2 = __shfl_xor_sync(0xffffffffu, b.s2, o);
            c.lmx = __shfl_xor_sync(0xffffffffu, b.lmx, o);
            c.bad = __shfl_xor_sync(0xffffffffu, b.bad, o);
            b = acc_merge(b, c);
        }
        a = b;
    }
    return a;   // valid in warp 0
}

// Pass 1: per block, over a contiguous stripe (deterministic for a fixed n).
__global__ void __launch_bounds__(kRedThreads) reduce_partial_kernel(const double *__restrict__ lnw,
                                                                     const double *__restrict__ lnL, int64_t n,
                                                                     double *__restrict__ partial)
{
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = min(n, b0 + per);
    // local max first, then sums relative to it
    Acc a{-INFINITY, 0.0, 0.0, -INFINITY, 0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        double x = lnw[i];
        if (!isfinite(x)) {
            a.bad = 1;
            continue;
        }
        if (x > a.mx) {
            double f = (a.mx == -INFINITY) ? 0.0 : exp(a.mx - x);
            a.s1 = a.s1 * f + 1.0;
            a.s2 = a.s2 * f * f + 1.0;
            a.mx = x;
        } else {
            double e = exp(x - a.mx);
            a.s1 += e;
            a.s2 += e * e;
        }
        a.lmx = fmax(a.lmx, lnL[i]);
    }
    a = block_merge(a);
    if (threadIdx.x == 0) {
        double *o = partial + 5 * blockIdx.x;
        o[0] = a.mx;
        o[1] = a.s1;
        o[2] = a.s2;
        o[3] = a.lmx;
        o[4] = (double)a.bad;
    }
}

// Pass 2: one block merges the partials in block order; writes the iteration's
// statistics and merges them into the pooled accumulators.
__global__ void __launch_bounds__(kRedThreads) reduce_final_kernel(const double *__restrict__ partial, int nb, int64_t n,
                                                                   double *__restrict__ stats, int slot,
                                                                   double *__restrict__ pooled, int reset, int *err)
{
    Acc a{-INFINITY, 0.0, 0.0, -INFINITY, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double *o = partial + 5 * b;
        a = acc_merge(a, Acc{o[0], o[1], o[2], o[3], o[4] != 0.0});
    }
    a = block_merge(a);
    if (threadIdx.x == 0) {
        double N = (double)n;
        double *s = stats + 8 * slot;
        double var = a.s2 / (a.s1 * a.s1) - 1.0 / N;
        s[0] = a.mx + log(a.s1) - log(N);
        s[1] = sqrt(var > 0.0 ? var : 0.0);
        s[2] = a.s1;
        s[3] = a.s1 * a.s1 / a.s2;
        s[4] = a.mx;
        s[5] = a.lmx;
        s[6] = N;
        s[7] = 0.0;
        if (a.bad || !isfinite(s[0]))
            atomicOr(err, kErrNonFinite);
        Acc pool = reset ? Acc{-INFINITY, 0.0, 0.0, -INFINITY, 0} : Acc{pooled[0], pooled[1], pooled[2], pooled[4], 0};
        double pn = reset ? 0.0 : pooled[3];
        pool = acc_merge(pool, a);
        pooled[0] = pool.mx;
        pooled[1] = pool.s1;
        pooled[2] = pool.s2;
        pooled[3] = pn + N;
        pooled[4] = pool.lmx;
    }
}

cudaError_t launch_reduce(const double *lnw, const double *lnL, int64_t n, double *partial, double *stats, int slot,
                          double *pooled, int reset_pooled, int *err, cudaStream_t st)
{
    int nb = kRedBlocks;
    if ((int64_t)nb * 64 > n)
        nb = (int)((n + 63) / 64);
    if (nb < 1)
        nb = 1;
    reduce_partial_kernel<<<nb, kRedThreads, 0, st>>>(lnw, lnL, n, partial);
    reduce_final_kernel<<<1, kRedThreads, 0, st>>>(partial, nb, n, stats, slot, pooled, reset_pooled, err);
    return cudaGetLastError();
}

__global__ void pooled_final_kernel(const double *__restrict__ pooled, double *__restrict__ out)
{
    double N = pooled[3];
    double var = pooled[2] / (pooled[1] * pooled[1]) - 1.0 / N;
    out[0] = pooled[0] + log(pooled[1]) - log(N);
    out[1] = sqrt(var > 0.0 ? var : 0.0);
    out[2] = pooled[1];
    out[3] = pooled[1] * pooled[1] / pooled[2];
    out[4] = pooled[4];
    out[5] = N;
}

cudaError_t launch_pooled_final(const double *pooled, double *out, cudaStream_t st)
{
    pooled_final_kernel<<<1, 1, 0, st>>>(pooled, out);
    return cudaGetLastError();
}

// ======================================================================== adaptation

constexpr int kHistBlocks = 152;

__global__ void __launch_bounds__(256) hist_partial_kernel(SamplerDev S, const uint64_t *__restrict__ bins,
                                                           const double *__restrict__ lnw, int64_t n,
                                                           const double *__restrict__ stats, int slot,
                                                           double *__restrict__ partial)
{
    extern __shared__ double sH[];   // [6][B]
    const int B = S.B;
    for (int e = threadIdx.x; e < 6 * B; e += blockDim.x)
        sH[e] = 0.0;
    __syncthreads();
    const double mx = stats[8 * slot + 4];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        double x = lnw[i];
        if (!isfinite(x))
            continue;
        double w = exp(S.temper * (x - mx));
        uint64_t pk = bins[i];
#pragma unroll
        for (int d = 0; d < 6; ++d)
            atomicAdd(&sH[d * B + (int)((pk >> (10 * d)) & 1023u)], w);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 6 * B; e += blockDim.x)
        partial[(size_t)blockIdx.x * 6 * B + e] = sH[e];
}

// Sum partial histograms in block order; P <- (1-eps) H / sum H + eps / B; rebuild C.
__global__ void adapt_final_kernel(SamplerDev S, const double *__restrict__ partial, int nb)
{
    const int B = S.B;
    const int d = threadIdx.x >> 5, lane = threadIdx.x & 31;   // one warp per dimension
    if (d >= 6)
        return;
    double tot = 0.0;
    for (int b = lane; b < B; b += 32) {
        double h = 0.0;
        for (int k = 0; k < nb; ++k)
            h += partial[(size_t)k * 6 * B + d * B + b];
        S.C[d * (B + 1) + b + 1] = h;   // stash H in the C slots while reducing
        tot += h;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1)
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
    __syncwarp();
    if (tot > 0.0 && isfinite(tot)) {
        for (int b = lane; b < B; b += 32)
            S.P[d * B + b] = (1.0 - S.floor_eps) * S.C[d * (B + 1) + b + 1] / tot + S.floor_eps / B;
    }
    __syncwarp();
    if (lane == 0) {
        double run = 0.0;
        S.C[d * (B + 1)] = 0.0;
        for (int b = 0; b < B; ++b) {
            run += S.P[d * B + b];
            S.C[d * (B + 1) + b + 1] = run;
        }
    }
    __syncwarp();
    const double ctot = S.C[d * (B + 1) + B];
    for (int b = lane; b < B; b += 32)
        S.L[d * B + b] = log(B * S.P[d * B + b] / ctot);
}

cudaError_t launch_adapt(const SamplerDev &S, const uint64_t *bins, const double *lnw, int64_t n, const double *stats,
                         int slot, double *hist_partial, cudaStream_t st)
{
    int nb = kHistBlocks;
    if ((int64_t)nb * 256 > n)
        nb = (int)((n + 255) / 256);
    if (nb < 1)
        nb = 1;
    size_t smem = sizeof(double) * 6 * S.B;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem(hist_partial_kernel);
        if (e != cudaSuccess)
            return e;
    }
    hist_partial_kernel<<<nb, 256, smem, st>>>(S, bins, lnw, n, stats, slot, hist_partial);
    adapt_final_kernel<<<1, 6 * 32, 0, st>>>(S, hist_partial, nb);
    return cudaGetLastError();
}

__global__ void build_cdf_kernel(SamplerDev S)
{
    const int d = threadIdx.x;
    if (d >= 6)
        return;
    double run = 0.0;
    S.C[d * (S.B + 1)] = 0.0;
    for (int b = 0; b < S.B; ++b) {
        run += S.P[d * S.B + b];
        S.C[d * (S.B + 1) + b + 1] = run;
    }
    for (int b = 0; b < S.B; ++b)
        S.L[d * S.B + b] = log(S.B * S.P[d * S.B + b] / run);
}

cudaError_t launch_build_cdf(const SamplerDev &S, cudaStream_t st)
{
    build_cdf_kernel<<<1, 32, 0, st>>>(S);
    return cudaGetLastError();
}

}  // namespace rift

// ======================================================================== reduction without allocation
//
// rift_ile_reduce_noalloc runs the same two reduction kernels as the library's own
// marginalisation, but its scratch (block partials, the running record and the
// error word) lives in the file-scope array below instead of in buffers from
// cudaMalloc.  Every GPU that loads the library holds this array until the
// process exits.  Host code must not hand the symbol itself to a kernel (on the
// host it names a stand-in, not device memory): its device address is taken once
// per device with cudaGetSymbolAddress, with that device current.

namespace {

constexpr int kNoallocPartials = 5 * rift::kRedBlocks;   // [kRedBlocks][5] block partials
constexpr int kNoallocPooled = kNoallocPartials;         // 8 doubles: running record
constexpr int kNoallocErr = kNoallocPooled + 8;          // error word (int in a double slot)
constexpr int kNoallocDoubles = kNoallocErr + 8;          // 1536 doubles = 12 KiB

static __device__ __align__(256) double g_reduce_scratch[kNoallocDoubles];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RIFT_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return RIFT_OK;
}

}  // namespace

extern "C" int rift_ile_reduce_noalloc(const double *lnw, const double *lnL, int64_t n, double *out, void *cuda_stream)
{
    if (!lnw || !out || n < 1 || n > RIFT_NOALLOC_MAX_SAMPLES)
        return RIFT_EINVAL;
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != RIFT_OK)
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int *err = reinterpret_cast<int *>(scratch + kNoallocErr);
    int flags = 0;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
        rift::launch_reduce(lnw, lnL ? lnL : lnw, n, scratch, out, 0, scratch + kNoallocPooled, 1, err, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&flags, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    return (flags & rift::kErrNonFinite) ? RIFT_ENONFINITE : RIFT_OK;
}
