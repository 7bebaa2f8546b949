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

#include "draws.cuh"
#include "ile_kernels.h"

namespace rift {

// ======================================================================== draw

constexpr int kDrawThreads = 256;

__global__ void __launch_bounds__(kDrawThreads) draw_kernel(SamplerDev S, SkyGrid G,
                                                            const uint32_t *__restrict__ iter_base, uint32_t iter_off,
                                                            int64_t n, double *__restrict__ theta,
                                                            double *__restrict__ lnpw, uint64_t *__restrict__ bins,
                                                            uint32_t *__restrict__ key)
{
    const uint32_t iter = *iter_base + iter_off;
    extern __shared__ double sC[];
    hist_load_tables(S, sC);
    __syncthreads();
    const uint32_t k0 = (uint32_t)S.seed, k1 = (uint32_t)(S.seed >> 32);
    const double d3lo = S.d_min * S.d_min * S.d_min, d3hi = S.d_max * S.d_max * S.d_max;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v[6], lr, th[6];
        uint64_t packed;
        hist_draw_one(sC, S.B, S.marg, iter, i, k0, k1, v, lr, packed);
        hist_theta(v, d3lo, d3hi, th);
        double *out = theta + 6 * i;
#pragma unroll
        for (int d = 0; d < 6; ++d)
            out[d] = th[d];
        lnpw[i] = lr;
        bins[i] = packed;
        // on the (right ascension, sin declination) grid the cell follows from the prior
        // coordinates themselves: alpha / 2 pi = v0 and (sin delta + 1) / 2 = v1
        key[i] = G.mode == kSortSky ? sky_cell_v(v[0], v[1], G) : sky_cell(th[0], th[1], G);
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

cudaError_t launch_draw(const SamplerDev &S, const SkyGrid &G, const uint32_t *iter_base, uint32_t iter_off, int64_t n,
                        double *theta, double *lnpw, uint64_t *bins, uint32_t *key, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    size_t smem = sizeof(double) * hist_table_doubles(S.B);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem(draw_kernel);
        if (e != cudaSuccess)
            return e;
    }
    draw_kernel<<<grid_for(n, kDrawThreads, 8), kDrawThreads, smem, st>>>(S, G, iter_base, iter_off, n, theta, lnpw, bins, key);
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

SkyGrid sky_grid_for(int64_t n, int per_cell)
{
    int order = 4;
    while (order < kMaxOrder && ((int64_t)per_cell << (2 * order)) < n)
        ++order;
    return SkyGrid{order, 1 << (2 * order)};
}

// ======================================================================== stable sort by sky cell
//
// Least-significant-digit radix sort of the cell keys (10-bit digits: one pass for
// grids of up to 1024 cells, two for up to 2^20), stable in the sample index: samples
// of one cell keep their draw order, so the tiles the likelihood kernels form, and
// with them every float32 result, are the same from run to run.  Each pass: per-tile
// digit counts (8192 samples per tile), an exclusive scan of the counts in
// digit-major order, and a scatter in which each warp walks its contiguous quarter of
// the tile in order and ranks equal digits with a warp match.

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixPerWarp = 1024;
constexpr int kRadixTile = kRadixWarps * kRadixPerWarp;

template <typename K>
__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const K *__restrict__ keys, int64_t n,
                                                                   int shift, int nblk, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[kRadixBuckets];
    for (int d = threadIdx.x; d < kRadixBuckets; d += kRadixThreads)
        h[d] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int j = threadIdx.x; j < kRadixTile; j += kRadixThreads) {
        const int64_t i = base + j;
        if (i < n)
            atomicAdd(&h[(uint32_t)(keys[i] >> shift) & (kRadixBuckets - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBuckets; d += kRadixThreads)
        hist[(size_t)d * nblk + blockIdx.x] = h[d];
}

template <typename K>
__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(const K *__restrict__ keys_in,
                                                                      const uint32_t *__restrict__ vals_in, int64_t n,
                                                                      int shift, int nblk,
                                                                      const uint32_t *__restrict__ offsets,
                                                                      K *__restrict__ keys_out,
                                                                      uint32_t *__restrict__ vals_out)
{
    __shared__ uint32_t wpos[kRadixWarps][kRadixBuckets];   // per-warp digit counts, then positions
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < kRadixWarps * kRadixBuckets; e += kRadixThreads)
        (&wpos[0][0])[e] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)w * kRadixPerWarp;
    for (int j = lane; j < kRadixPerWarp; j += 32) {
        const int64_t i = base + j;
        if (i < n)
            atomicAdd(&wpos[w][(uint32_t)(keys_in[i] >> shift) & (kRadixBuckets - 1)], 1u);
    }
    __syncthreads();
    // first position of each digit for each warp: the tile's offset, then warps in order
    for (int d = threadIdx.x; d < kRadixBuckets; d += kRadixThreads) {
        uint32_t run = offsets[(size_t)d * nblk + blockIdx.x];
#pragma unroll
        for (int v = 0; v < kRadixWarps; ++v) {
            const uint32_t c = wpos[v][d];
            wpos[v][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int j0 = 0; j0 < kRadixPerWarp && base + j0 < n; j0 += 32) {
        const int64_t i = base + j0 + lane;
        const bool ok = i < n;
        const K k = ok ? keys_in[i] : (K)0;
        const uint32_t d = ok ? (uint32_t)(k >> shift) & (kRadixBuckets - 1) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok) {
            const uint32_t pos = wpos[w][d] + __popc(peers & ((1u << lane) - 1u));
            if (vals_out)
                vals_out[pos] = vals_in ? vals_in[i] : (uint32_t)i;
            if (keys_out)
                keys_out[pos] = k;
        }
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1)
            wpos[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

// Exclusive scan of L counts in place: per-tile totals of 4096 counts, a scan of the
// totals (recursively when there are more than 1024 tiles), then a block-level scan
// of each tile offset by its total.  Coalesced loads and stores; each thread owns 16
// consecutive counts staged through shared memory.  32-bit for the sort, 64-bit for
// the fair draws' fixed-point weights.
constexpr int kScanTile = 4096;
constexpr int kScanThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_totals_kernel(const T *__restrict__ counts, int n_cells,
                                                                   T *__restrict__ totals)
{
    __shared__ T red[kScanThreads / 32];
    const int base = blockIdx.x * kScanTile;
    T v = 0;
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
        T t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w)
            t += red[w];
        totals[blockIdx.x] = t;
    }
}

// Block-wide exclusive scan of one value per thread; returns this thread's offset.
template <typename T> __device__ T block_exclusive_scan(T v, T *warp_tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return x - v + (w > 0 ? warp_tot[w - 1] : (T)0);
}

template <typename T> __global__ void __launch_bounds__(1024) scan_top_kernel(T *totals, int nb)
{
    __shared__ T warp_tot[32];
    const T v = threadIdx.x < nb ? totals[threadIdx.x] : (T)0;
    const T e = block_exclusive_scan(v, warp_tot);
    if (threadIdx.x < nb)
        totals[threadIdx.x] = e;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(T *__restrict__ counts, int n_cells,
                                                                  const T *__restrict__ totals)
{
    constexpr int per = kScanTile / kScanThreads;
    __shared__ T tile[kScanTile + kScanTile / 32];   // padded: thread-strided reads avoid conflicts
    __shared__ T warp_tot[32];
    const int base = blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        tile[i + (i >> 5)] = base + i < n_cells ? counts[base + i] : (T)0;
    __syncthreads();
    T loc[per], run = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int i = threadIdx.x * per + q;
        loc[q] = run;
        run += tile[i + (i >> 5)];
    }
    const T off = block_exclusive_scan(run, warp_tot) + totals[blockIdx.x];
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

// Exclusive scan of data[0, L) in place; scratch holds the totals of every level.
template <typename T> static int launch_scan(T *data, int L, T *scratch, cudaStream_t st)
{
    const int nb = (L + kScanTile - 1) / kScanTile;
    scan_totals_kernel<T><<<nb, kScanThreads, 0, st>>>(data, L, scratch);
    int launched = 1;
    if (nb <= 1024) {
        scan_top_kernel<T><<<1, 1024, 0, st>>>(scratch, nb);
        ++launched;
    } else {
        launched += launch_scan<T>(scratch, nb, scratch + nb, st);
    }
    scan_apply_kernel<T><<<nb, kScanThreads, 0, st>>>(data, L, scratch);
    return launched + 1;
}

size_t scan_scratch_words(int64_t L)
{
    size_t words = 0;
    while (L > 1) {
        L = (L + kScanTile - 1) / kScanTile;
        words += (size_t)L;
    }
    return words + 1;
}

cudaError_t launch_scan_u64(uint64_t *data, int64_t L, uint64_t *scratch, cudaStream_t st, int *launched)
{
    const int k = L > 0 ? launch_scan<uint64_t>(data, (int)L, scratch, st) : 0;
    if (launched)
        *launched = k;
    return cudaGetLastError();
}

size_t sort_scratch_words(int64_t n_max)
{
    const int64_t nblk = (n_max + kRadixTile - 1) / kRadixTile;
    int64_t L = (int64_t)kRadixBuckets * (nblk > 0 ? nblk : 1), words = L;
    while (L > 1) {   // totals of every scan level
        L = (L + kScanTile - 1) / kScanTile;
        words += L;
    }
    return (size_t)(words + 2 * n_max + 64);
}

cudaError_t launch_sort(const SkyGrid &G, const uint32_t *key, int64_t n, uint32_t *scratch, uint32_t *perm,
                        cudaStream_t st, int *launched)
{
    if (launched)
        *launched = 0;
    if (n <= 0)
        return cudaSuccess;
    const int nblk = (int)((n + kRadixTile - 1) / kRadixTile);
    const int L = kRadixBuckets * nblk;
    uint32_t *hist = scratch;
    uint32_t *key_tmp = hist + L, *val_tmp = key_tmp + n;
    uint32_t *scan_scratch = val_tmp + n;
    const int passes = G.n_cells <= kRadixBuckets ? 1 : 2;
    int count = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kRadixBits;
        const bool last = pass == passes - 1;
        const uint32_t *kin = pass == 0 ? key : key_tmp;
        const uint32_t *vin = pass == 0 ? nullptr : val_tmp;
        radix_hist_kernel<uint32_t><<<nblk, kRadixThreads, 0, st>>>(kin, n, shift, nblk, hist);
        count += 1 + launch_scan<uint32_t>(hist, L, scan_scratch, st);
        radix_scatter_kernel<uint32_t><<<nblk, kRadixThreads, 0, st>>>(kin, vin, n, shift, nblk, hist,
                                                                       last ? nullptr : key_tmp, last ? perm : val_tmp);
        count += 1;
    }
    if (launched)
        *launched = count;
    return cudaGetLastError();
}

size_t sort64_scratch_words(int64_t n_max)
{
    const int64_t nblk = (n_max + kRadixTile - 1) / kRadixTile;
    int64_t L = (int64_t)kRadixBuckets * (nblk > 0 ? nblk : 1), words = L;
    while (L > 1) {
        L = (L + kScanTile - 1) / kScanTile;
        words += L;
    }
    return (size_t)(words + 64);
}

cudaError_t launch_sort64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, uint32_t *scratch, cudaStream_t st,
                          int *launched)
{
    if (launched)
        *launched = 0;
    if (n <= 0)
        return cudaSuccess;
    const int nblk = (int)((n + kRadixTile - 1) / kRadixTile);
    const int L = kRadixBuckets * nblk;
    uint32_t *hist = scratch, *scan_scratch = scratch + L;
    const int passes = bits <= 0 ? 0 : (bits + kRadixBits - 1) / kRadixBits;
    int count = 0;
    uint64_t *in = keys, *out = tmp;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kRadixBits;
        radix_hist_kernel<uint64_t><<<nblk, kRadixThreads, 0, st>>>(in, n, shift, nblk, hist);
        count += 1 + launch_scan<uint32_t>(hist, L, scan_scratch, st);
        radix_scatter_kernel<uint64_t><<<nblk, kRadixThreads, 0, st>>>(in, nullptr, n, shift, nblk, hist, out,
                                                                       nullptr);
        count += 1;
        uint64_t *t = in;
        in = out;
        out = t;
    }
    if (in != keys) {   // odd number of passes: the sorted keys are in tmp
        cudaError_t e = cudaMemcpyAsync(keys, in, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess)
            return e;
    }
    if (launched)
        *launched = count;
    return cudaGetLastError();
}

cudaError_t launch_scan_u32(uint32_t *data, int64_t L, uint32_t *scratch, cudaStream_t st, int *launched)
{
    const int k = L > 0 ? launch_scan<uint32_t>(data, (int)L, scratch, st) : 0;
    if (launched)
        *launched = k;
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

// exp(t) for t <= 0: float64, or float32 for terms that carry float32 errors already
// (float64 exponentials run on this part's slow float64 pipe)
__device__ __forceinline__ double term_exp(double t, bool f32)
{
    return f32 ? (double)expf((float)t) : exp(t);
}

// Pass 1: per block, over a contiguous stripe (deterministic for a fixed n).
__global__ void __launch_bounds__(kRedThreads) reduce_partial_kernel(const double *__restrict__ lnw,
                                                                     const double *__restrict__ lnL, int64_t n,
                                                                     double *__restrict__ partial, bool f32)
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
            double f = (a.mx == -INFINITY) ? 0.0 : term_exp(a.mx - x, f32);
            a.s1 = a.s1 * f + 1.0;
            a.s2 = a.s2 * f * f + 1.0;
            a.mx = x;
        } else {
            double e = term_exp(x - a.mx, f32);
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
                          double *pooled, int reset_pooled, int *err, cudaStream_t st, bool f32_terms)
{
    int nb = kRedBlocks;
    if ((int64_t)nb * 64 > n)
        nb = (int)((n + 63) / 64);
    if (nb < 1)
        nb = 1;
    reduce_partial_kernel<<<nb, kRedThreads, 0, st>>>(lnw, lnL, n, partial, f32_terms);
    reduce_final_kernel<<<1, kRedThreads, 0, st>>>(partial, nb, n, stats, slot, pooled, reset_pooled, err);
    return cudaGetLastError();
}

__global__ void pooled_final_kernel(const double *__restrict__ pooled, double *__restrict__ out, uint32_t *iter_base,
                                    uint32_t advance)
{
    *iter_base += advance;
    double N = pooled[3];
    double var = pooled[2] / (pooled[1] * pooled[1]) - 1.0 / N;
    out[0] = pooled[0] + log(pooled[1]) - log(N);
    out[1] = sqrt(var > 0.0 ? var : 0.0);
    out[2] = pooled[1];
    out[3] = pooled[1] * pooled[1] / pooled[2];
    out[4] = pooled[4];
    out[5] = N;
}

cudaError_t launch_pooled_final(const double *pooled, double *out, uint32_t *iter_base, uint32_t advance,
                                cudaStream_t st)
{
    pooled_final_kernel<<<1, 1, 0, st>>>(pooled, out, iter_base, advance);
    return cudaGetLastError();
}

// ======================================================================== adaptation

constexpr int kHistBlocks = 152;

// Histogram weights are summed exactly, in 128-bit fixed point with 2^-90 resolution
// (lo, hi words): integer addition does not depend on the order in which samples
// arrive, so the adapted sampler is bitwise reproducible however the blocks and
// atomics interleave (and a solve's result does not depend on what else runs).
// Weights are w = exp(beta (ln w_i - max ln w)) <= 1; at most 2^31 samples keep the
// sum below 2^121.
constexpr int kFixShift = 90;

__device__ __forceinline__ void to_fixed(double w, uint64_t &lo, uint64_t &hi)
{
    lo = hi = 0;
    if (!(w > 0.0))
        return;
    w = fmin(w, 1.0);
    const uint64_t bits = (uint64_t)__double_as_longlong(w);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    if (e < -kFixShift - 1)
        return;
    const uint64_t m = (bits & ((1ull << 52) - 1)) | (1ull << 52);   // w = m 2^(e-52)
    const int s = e - 52 + kFixShift;                                  // W = m 2^s
    if (s >= 64) {
        hi = m << (s - 64);
    } else if (s > 0) {
        lo = m << s;
        hi = m >> (64 - s);
    } else if (s > -64) {
        lo = m >> (-s);
    }
}

__device__ __forceinline__ void add_fixed(unsigned long long *lo, unsigned long long *hi, uint64_t a_lo, uint64_t a_hi)
{
    if (a_lo) {
        const unsigned long long old = atomicAdd(lo, (unsigned long long)a_lo);
        if (old + a_lo < old)
            ++a_hi;   // this addition wrapped the low word
    }
    if (a_hi)
        atomicAdd(hi, (unsigned long long)a_hi);
}

__global__ void __launch_bounds__(256) hist_partial_kernel(SamplerDev S, const uint64_t *__restrict__ bins,
                                                           const double *__restrict__ lnw, int64_t n,
                                                           const double *__restrict__ stats, int slot,
                                                           uint64_t *__restrict__ partial, bool f32)
{
    extern __shared__ unsigned long long sF[];   // [6][B][2] = (lo, hi) per bin
    const int B = S.B;
    for (int e = threadIdx.x; e < 12 * B; e += blockDim.x)
        sF[e] = 0ull;
    __syncthreads();
    const double mx = stats[8 * slot + 4];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        double x = lnw[i];
        if (!isfinite(x))
            continue;
        uint64_t lo, hi;
        to_fixed(term_exp(S.temper * (x - mx), f32), lo, hi);
        if (!(lo | hi))
            continue;
        uint64_t pk = bins[i];
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const int e = d * B + (int)((pk >> (10 * d)) & 1023u);
            add_fixed(&sF[2 * e], &sF[2 * e + 1], lo, hi);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 12 * B; e += blockDim.x)
        partial[(size_t)blockIdx.x * 12 * B + e] = sF[e];
}

// Sum the partial histograms exactly (128-bit); P <- (1-eps) H / sum H + eps / B; rebuild C.
// One block per dimension: the bins' sums over the block partials are split across the
// block's threads (integer sums, so the same H in any split), then one warp finishes.
constexpr int kAdaptFinalThreads = 256;
__global__ void __launch_bounds__(kAdaptFinalThreads) adapt_final_kernel(SamplerDev S,
                                                                         const uint64_t *__restrict__ partial, int nb)
{
    const int B = S.B, d = blockIdx.x;
    if (d >= 6 || (S.marg && d == 5))   // a marginalised distance keeps its masses
        return;
    __shared__ unsigned long long acc[3][kAdaptFinalThreads];
    const int tpb = B < kAdaptFinalThreads ? kAdaptFinalThreads / B : 1;   // threads per bin
    const int t = threadIdx.x, j = t % tpb, b0 = t / tpb, bstride = kAdaptFinalThreads / tpb;
    for (int bb = 0; bb < B; bb += bstride) {
        const int b = bb + b0;
        const bool mine = b0 < bstride && b < B;
        // the low words are summed as two 32-bit halves (no carry chain between the
        // loads), then recombined exactly
        uint64_t l0 = 0, l1 = 0, hi = 0;
        if (mine) {
#pragma unroll 4
            for (int k = j; k < nb; k += tpb) {
                const uint64_t *q = partial + (size_t)k * 12 * B + 2 * (d * B + b);
                const uint64_t lo = q[0];
                l0 += lo & 0xffffffffull;
                l1 += lo >> 32;
                hi += q[1];
            }
        }
        acc[0][t] = l0;
        acc[1][t] = l1;
        acc[2][t] = hi;
        __syncthreads();
        if (mine && j == 0) {
            for (int u = 1; u < tpb; ++u) {
                l0 += acc[0][t + u];
                l1 += acc[1][t + u];
                hi += acc[2][t + u];
            }
            const uint64_t a = l0 + (l1 << 32);
            hi += (l1 >> 32) + (a < l0 ? 1u : 0u);
            S.C[d * (B + 1) + b + 1] = ldexp((double)hi, 64 - kFixShift) + ldexp((double)a, -kFixShift);   // H
        }
        __syncthreads();
    }
    if (t >= 32)
        return;
    const int lane = t;
    double tot = 0.0;
    for (int b = lane; b < B; b += 32)
        tot += S.C[d * (B + 1) + b + 1];   // H stashed in the C slots while reducing
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
                         int slot, uint64_t *hist_partial, cudaStream_t st, bool f32_terms)
{
    int nb = kHistBlocks;
    if ((int64_t)nb * 256 > n)
        nb = (int)((n + 255) / 256);
    if (nb < 1)
        nb = 1;
    size_t smem = sizeof(uint64_t) * 12 * S.B;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem(hist_partial_kernel);
        if (e != cudaSuccess)
            return e;
    }
    hist_partial_kernel<<<nb, 256, smem, st>>>(S, bins, lnw, n, stats, slot, hist_partial, f32_terms);
    adapt_final_kernel<<<6, kAdaptFinalThreads, 0, st>>>(S, hist_partial, nb);
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

cudaError_t prepare_sampler_kernels()
{
    cudaError_t e = allow_max_dynamic_smem(draw_kernel);
    return e != cudaSuccess ? e : allow_max_dynamic_smem(hist_partial_kernel);
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
