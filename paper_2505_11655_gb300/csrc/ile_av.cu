// Adaptive-volume (AV) integrator on the device (include/rift_ile.h, rift_ile_av):
// arXiv:2505.11655, Sec. IV A.
//
// The unit cube of prior-CDF coordinates v (the prior is uniform there, Z = int L dv)
// is covered by nested grids of 2^level cells per side; a sorted list of active cell
// keys (coordinate d of a cell in bits [level d, level (d+1))) defines the sampling
// region.  One iteration:
//   1. n draws uniform over the active cells (sampling density 1/V, ln w = ln L + ln V);
//   2. the time-marginalised ln L of the draws (the same kernels as every other path);
//   3. fresh points that pass the current threshold join the live set (index order,
//      up to its capacity);
//   4. threshold: a 1/64-wide ln L histogram below the live maximum m with exact
//      fixed-point masses floor(exp(ln L - m) 2^S), S = 62 - ceil(log2 N_live); the kept
//      bins are the fewest from the top holding both the fraction P_thr of the mass and
//      at least N_min* points (decided on the host in integers).  N_min* is a floor: while
//      the likelihood is poorly resolved a handful of points carry P_thr of the mass, and
//      the top N_min* points set the threshold, beyond the histogram's range when need be
//      (the N_min*-th smallest bin index, from a sort of every live point's bin);
//   5. refine: with V_thr the estimated volume above the current threshold (1 at the
//      start; the live points are uniform in that region), V' = V_thr N_min / N_live,
//      dV = V' / sqrt(N_min), n_bins = (1/dV)^(1/6) (Eq. nbins_V) rounded down to a power
//      of two, never coarser; V_thr <- V'.  The new active cells are those holding a kept
//      live point (64-bit radix sort of the cell keys, unique); draws are uniform over
//      them (volume V >= V_thr).
#include <cmath>
#include <cstring>
#include <vector>

#include "draws.cuh"
#include "ile_handle.h"

using namespace rift;
using namespace rift::host;

namespace {

constexpr int kAvBinsPerUnit = 64;
constexpr int kAvHist = 4096;
constexpr int kAvMaxLevel = 10;
constexpr int kAvHistBlocks = 152;
constexpr int kAvPShift = 20;

__global__ void av_draw_kernel(const uint64_t *__restrict__ cells, int64_t n_cells, int level, uint64_t seed,
                               uint32_t iter, int64_t n, double d_min, double d_max, double lnV,
                               double *__restrict__ theta, double *__restrict__ lnpw, double *__restrict__ v_out)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double d3lo = d_min * d_min * d_min, d3hi = d_max * d_max * d_max;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v[6];
        av_draw_one(cells, n_cells, level, iter, i, k0, k1, v);
#pragma unroll
        for (int d = 0; d < 6; ++d)
            v_out[6 * i + d] = v[d];
        av_theta(v, d3lo, d3hi, theta + 6 * i);
        lnpw[i] = lnV;
    }
}

__device__ __forceinline__ bool av_passes(double lnL, bool has_thr, double m, int64_t b)
{
    return !has_thr || floor(__dmul_rn(__dsub_rn(m, lnL), (double)kAvBinsPerUnit)) <= (double)b;
}

// flags[i] = point i passes; flags[n] = 0 (so that the exclusive scan ends in the total)
__global__ void av_flags_kernel(const double *__restrict__ lnL, int64_t n, bool has_thr, double m, int64_t b,
                                uint32_t *__restrict__ flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = i < n && av_passes(lnL[i], has_thr, m, b) ? 1u : 0u;
}

// points that pass go to dst[base + rank] while rank < room
__global__ void av_scatter_kernel(const double *__restrict__ v, const double *__restrict__ lnL, int64_t n,
                                  bool has_thr, double m, int64_t b, const uint32_t *__restrict__ rank, int64_t base,
                                  int64_t room, double *__restrict__ v_dst, double *__restrict__ lnL_dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!av_passes(lnL[i], has_thr, m, b))
            continue;
        const int64_t r = rank[i];
        if (r >= room)
            continue;
        const int64_t o = base + r;
#pragma unroll
        for (int d = 0; d < 6; ++d)
            v_dst[6 * o + d] = v[6 * i + d];
        lnL_dst[o] = lnL[i];
    }
}

__device__ __forceinline__ unsigned long long order_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double from_order_bits(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

__global__ void av_max_kernel(const double *__restrict__ lnL, int64_t n, unsigned long long *out)
{
    unsigned long long best = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (isfinite(lnL[i]))
            best = max(best, order_bits(lnL[i]));
#pragma unroll
    for (int o = 16; o; o >>= 1)
        best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best)
        atomicMax(out, best);
}

// per-block exact histograms of the live ln L (bins of 1/64 below the maximum)
__global__ void __launch_bounds__(256) av_hist_kernel(const double *__restrict__ lnL, int64_t n,
                                                      const unsigned long long *__restrict__ maxbits, int S,
                                                      uint64_t *__restrict__ mass_part,
                                                      uint32_t *__restrict__ count_part)
{
    extern __shared__ unsigned long long sM[];   // [kAvHist] masses, then [kAvHist] counts (as u32)
    uint32_t *sC = reinterpret_cast<uint32_t *>(sM + kAvHist);
    for (int e = threadIdx.x; e < kAvHist; e += blockDim.x) {
        sM[e] = 0ull;
        sC[e] = 0u;
    }
    __syncthreads();
    const double m = from_order_bits(*maxbits);
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double x = lnL[i];
        if (!isfinite(x))
            continue;
        const double bf = floor(__dmul_rn(__dsub_rn(m, x), (double)kAvBinsPerUnit));
        if (!(bf < (double)kAvHist))
            continue;
        const int b = (int)bf;
        atomicAdd(&sM[b], (unsigned long long)(uint64_t)ldexp(exp(x - m), S));
        atomicAdd(&sC[b], 1u);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kAvHist; e += blockDim.x) {
        mass_part[(size_t)blockIdx.x * kAvHist + e] = sM[e];
        count_part[(size_t)blockIdx.x * kAvHist + e] = sC[e];
    }
}

__global__ void av_hist_final_kernel(const uint64_t *__restrict__ mass_part, const uint32_t *__restrict__ count_part,
                                     int nb, uint64_t *__restrict__ mass, uint32_t *__restrict__ count)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kAvHist)
        return;
    uint64_t mm = 0;
    uint32_t cc = 0;
    for (int k = 0; k < nb; ++k) {
        mm += mass_part[(size_t)k * kAvHist + e];
        cc += count_part[(size_t)k * kAvHist + e];
    }
    mass[e] = mm;
    count[e] = cc;
}

// bin index floor((m - ln L) 64) of every live point as a sort key (non-finite values and
// bins beyond 2^40 - 1 take the largest key)
constexpr int kAvBinKeyBits = 40;
__global__ void av_bin_keys_kernel(const double *__restrict__ lnL, int64_t n,
                                   const unsigned long long *__restrict__ maxbits, uint64_t *__restrict__ keys)
{
    const double m = from_order_bits(*maxbits);
    const uint64_t kmax = (1ull << kAvBinKeyBits) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = lnL[i];
        const double bf = isfinite(x) ? floor(__dmul_rn(__dsub_rn(m, x), (double)kAvBinsPerUnit)) : (double)kmax;
        keys[i] = bf < (double)kmax ? (uint64_t)bf : kmax;
    }
}

__global__ void av_keys_kernel(const double *__restrict__ v, int64_t n, int level, uint64_t *__restrict__ keys)
{
    const double side = ldexp(1.0, level);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
#pragma unroll
        for (int d = 0; d < 6; ++d)
            k |= (uint64_t)floor(__dmul_rn(v[6 * i + d], side)) << (level * d);
        keys[i] = k;
    }
}

// flags[i] = first occurrence of keys[i] in the sorted list; flags[n] = 0
__global__ void av_unique_flags_kernel(const uint64_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = i < n && (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void av_unique_scatter_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                         const uint32_t *__restrict__ rank, uint64_t *__restrict__ cells)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || keys[i] != keys[i - 1])
            cells[rank[i]] = keys[i];
}

int grid1(int64_t n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256, cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

int ceil_log2(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n)
        ++c;
    return c;
}

}  // namespace

namespace rift {
namespace host {

int av_alloc(rift_ile_t *h, int64_t cap)
{
    auto &a = h->av;
    const int64_t N = h->cap, F = std::max(cap, N) + 1;
    int rc;
    if ((rc = dalloc(h, &a.v, (size_t)cap * 6)) || (rc = dalloc(h, &a.lnL, (size_t)cap)) ||
        (rc = dalloc(h, &a.v2, (size_t)cap * 6)) || (rc = dalloc(h, &a.lnL2, (size_t)cap)) ||
        (rc = dalloc(h, &a.v_fresh, (size_t)N * 6)) || (rc = dalloc(h, &a.cells, (size_t)cap)) ||
        (rc = dalloc(h, &a.keys, (size_t)cap)) || (rc = dalloc(h, &a.keys_tmp, (size_t)cap)) ||
        (rc = dalloc(h, &a.flags, (size_t)F)) || (rc = dalloc(h, &a.scan, scan_scratch_words(F))) ||
        (rc = dalloc(h, &a.sort, sort64_scratch_words(cap))) ||
        (rc = dalloc(h, &a.mass_part, (size_t)kAvHistBlocks * kAvHist)) ||
        (rc = dalloc(h, &a.count_part, (size_t)kAvHistBlocks * kAvHist)) ||
        (rc = dalloc(h, &a.mass, (size_t)kAvHist)) || (rc = dalloc(h, &a.count, (size_t)kAvHist)) ||
        (rc = dalloc(h, &a.maxbits, (size_t)1)))
        return rc;
    CK(allow_max_dynamic_smem(av_hist_kernel));
    a.cap = cap;
    return RIFT_OK;
}

int av_restart(rift_ile_t *h)
{
    auto &a = h->av;
    a.level = 0;
    a.n_cells = 1;
    a.V = 1.0;
    a.V_thr = 1.0;
    a.n_live = 0;
    a.has_thr = false;
    a.iter = 0;
    CK(cudaMemsetAsync(a.cells, 0, sizeof(uint64_t), h->stream));
    return RIFT_OK;
}

}  // namespace host
}  // namespace rift

namespace {

// Exclusive scan of flags[0..n] in place and the total (flags[n] after the scan).
int scan_total(rift_ile_t *h, int64_t n, int64_t *total)
{
    auto &a = h->av;
    int k = 0;
    CK(launch_scan_u32(a.flags, n + 1, a.scan, h->stream, &k));
    uint32_t t = 0;
    CK(cudaMemcpyAsync(&t, a.flags + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *total = t;
    h->launches += k;
    return RIFT_OK;
}

int av_iteration(rift_ile_t *h, int64_t n, int slot, bool reset_pooled, double p_thr, int64_t n_min_star)
{
    auto &a = h->av;
    cudaStream_t st = h->stream;
    // 1. draw
    CK(mark(h, slot, 0));
    av_draw_kernel<<<grid1(n), 256, 0, st>>>(a.cells, a.n_cells, a.level, h->cfg.seed, a.iter, n, h->cfg.d_min_mpc,
                                             h->cfg.d_max_mpc, std::log(a.V), h->theta, h->lnpw, a.v_fresh);
    CK(cudaGetLastError());
    int sorted = 0;
    if (use_fp32(h)) {
        RK(grid_for_batch(h, n));
        CK(launch_keys(h->grid, h->theta, n, h->key, st));
        CK(launch_sort(h->grid, h->key, n, h->sort_scratch, h->perm, st, &sorted));
        sorted += 1;
    }
    CK(mark(h, slot, 1));
    // 2. likelihood
    if (!use_fp32(h)) {
        CK(launch_lnl_fp64(h->prob, h->theta, n, h->lnL, nullptr, h->lnpw, h->lnw, h->err, st));
    } else {
        CK(launch_tiled(h, h->theta, n, h->lnL, nullptr, h->lnpw, h->lnw));
        if (h->cfg.precision == RIFT_MIXED)
            RK(refine_batch(h, h->theta, n, h->lnL, h->lnpw, h->lnw));
    }
    CK(mark(h, slot, 2));
    CK(launch_reduce(h->lnw, h->lnL, n, h->red_partial, h->stats, slot, h->pooled, reset_pooled ? 1 : 0, h->err,
                     st, h->cfg.precision == RIFT_FP32));
    CK(mark(h, slot, 3));
    h->launches += 1 + sorted + 1 + 2;
    return av_update(h, a.v_fresh, h->lnL, n, p_thr, n_min_star);
}

}  // namespace

namespace rift {
namespace host {

int av_update(rift_ile_t *h, const double *v_fresh, const double *lnL_fresh, int64_t n, double p_thr,
              int64_t n_min_star)
{
    auto &a = h->av;
    cudaStream_t st = h->stream;
    // 3. live set
    av_flags_kernel<<<grid1(n + 1), 256, 0, st>>>(lnL_fresh, n, a.has_thr, a.m, a.b, a.flags);
    int64_t passed = 0;
    RK(scan_total(h, n, &passed));
    const int64_t room = a.cap - a.n_live;
    av_scatter_kernel<<<grid1(n), 256, 0, st>>>(v_fresh, lnL_fresh, n, a.has_thr, a.m, a.b, a.flags, a.n_live, room,
                                                a.v, a.lnL);
    CK(cudaGetLastError());
    a.n_live += std::min(passed, room);
    const int64_t n_live = a.n_live;
    // 4. threshold
    CK(cudaMemsetAsync(a.maxbits, 0, sizeof(unsigned long long), st));
    av_max_kernel<<<grid1(n_live), 256, 0, st>>>(a.lnL, n_live, a.maxbits);
    const int S = 62 - ceil_log2(n_live);
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kAvHistBlocks, (n_live + 255) / 256));
    av_hist_kernel<<<nb, 256, kAvHist * 12, st>>>(a.lnL, n_live, a.maxbits, S, a.mass_part, a.count_part);
    av_hist_final_kernel<<<kAvHist / 256, 256, 0, st>>>(a.mass_part, a.count_part, nb, a.mass, a.count);
    h->launches += 6;
    std::vector<uint64_t> mass(kAvHist);
    std::vector<uint32_t> count(kAvHist);
    unsigned long long mbits = 0;
    CK(cudaMemcpyAsync(mass.data(), a.mass, sizeof(uint64_t) * kAvHist, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(count.data(), a.count, sizeof(uint32_t) * kAvHist, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&mbits, a.maxbits, sizeof(mbits), cudaMemcpyDeviceToHost, st));
    RK(sync_and_err(h));
    if (mbits == 0)
        return RIFT_ENONFINITE;
    uint64_t bits = (mbits >> 63) ? (mbits & 0x7fffffffffffffffull) : ~mbits;
    double m;
    std::memcpy(&m, &bits, sizeof(m));
    unsigned __int128 total = 0;
    for (int e = 0; e < kAvHist; ++e)
        total += mass[e];
    const uint64_t p_num = (uint64_t)std::floor(p_thr * (double)(1u << kAvPShift));
    const int64_t need = std::min<int64_t>(n_min_star, n_live);
    unsigned __int128 run_m = 0;
    int64_t run_c = 0;
    int64_t b_mass = -1, b_count = -1;
    for (int e = 0; e < kAvHist && (b_mass < 0 || b_count < 0); ++e) {
        run_m += mass[e];
        run_c += count[e];
        if (b_mass < 0 && (run_m << kAvPShift) >= (unsigned __int128)p_num * total)
            b_mass = e;
        if (b_count < 0 && run_c >= need)
            b_count = e;
    }
    if (b_count < 0 && need > 0) {
        // the need-th largest value lies beyond the histogram's range: its bin, the need-th
        // smallest bin index of the live points
        av_bin_keys_kernel<<<grid1(n_live), 256, 0, st>>>(a.lnL, n_live, a.maxbits, a.keys);
        int ks = 0;
        CK(launch_sort64(a.keys, a.keys_tmp, n_live, kAvBinKeyBits, a.sort, st, &ks));
        uint64_t kb = 0;
        CK(cudaMemcpyAsync(&kb, a.keys + (need - 1), sizeof(kb), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        b_count = (int64_t)kb;
        h->launches += 1 + ks;
    }
    const int64_t b_thr = std::max<int64_t>(b_mass < 0 ? kAvHist - 1 : b_mass, b_count);
    av_flags_kernel<<<grid1(n_live + 1), 256, 0, st>>>(a.lnL, n_live, true, m, b_thr, a.flags);
    int64_t kept = 0;
    RK(scan_total(h, n_live, &kept));
    const int64_t n_min = kept;
    // 5. refine
    const double v_next = a.V_thr * (double)n_min / (double)n_live;
    const double dV = v_next / std::sqrt((double)n_min);
    const double nbins = std::pow(1.0 / dV, 1.0 / 6.0);
    const int cand = nbins >= 1.0 ? (int)std::floor(std::log2(nbins)) : 0;
    const int level = std::max(a.level, std::min(kAvMaxLevel, cand));
    a.V_thr = v_next;
    av_scatter_kernel<<<grid1(n_live), 256, 0, st>>>(a.v, a.lnL, n_live, true, m, b_thr, a.flags, 0, kept, a.v2,
                                                     a.lnL2);
    std::swap(a.v, a.v2);
    std::swap(a.lnL, a.lnL2);
    a.n_live = kept;
    av_keys_kernel<<<grid1(kept), 256, 0, st>>>(a.v, kept, level, a.keys);
    int k = 0;
    CK(launch_sort64(a.keys, a.keys_tmp, kept, 6 * level, a.sort, st, &k));
    av_unique_flags_kernel<<<grid1(kept + 1), 256, 0, st>>>(a.keys, kept, a.flags);
    int64_t ncells = 0;
    RK(scan_total(h, kept, &ncells));
    av_unique_scatter_kernel<<<grid1(kept), 256, 0, st>>>(a.keys, kept, a.flags, a.cells);
    CK(cudaGetLastError());
    h->launches += 6 + k;
    a.level = level;
    a.n_cells = ncells;
    a.V = std::ldexp((double)ncells, -6 * level);
    a.has_thr = true;
    a.m = m;
    a.b = b_thr;
    a.iter += 1;
    return RIFT_OK;
}

}  // namespace host
}  // namespace rift

extern "C" {

int rift_ile_av(rift_ile_t *h, int32_t n_iter, int64_t n_per_iter, double p_thr, int64_t n_min_star,
                int64_t capacity, int32_t restart, rift_ile_result *out)
{
    if (!h || h->cfg.distance_marg || n_iter < 1 || n_iter > RIFT_MAX_ITER || n_per_iter < 1 || n_per_iter > h->cap || !(p_thr > 0.0) ||
        !(p_thr <= 1.0) || n_min_star < 1 || capacity < n_per_iter || capacity > ((int64_t)1 << 31) - 2)
        return RIFT_EINVAL;
    if (!h->have_overlaps)
        return RIFT_ESTATE;
    if (h->av.cap != 0 && h->av.cap != capacity)
        return RIFT_EINVAL;   // the live-set capacity is fixed by the first call
    if (h->av.cap == 0) {
        RK(av_alloc(h, capacity));
        RK(av_restart(h));
    } else if (restart) {
        RK(av_restart(h));
    }
    RK(choose_plan(h, n_per_iter));
    RK(ensure_events(h, n_iter));
    h->timed = true;
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    for (int g = 0; g < n_iter; ++g)
        RK(av_iteration(h, n_per_iter, g, g == 0, p_thr, n_min_star));
    CK(launch_pooled_final(h->pooled, h->final_out, h->iter_dev, 0u, h->stream));
    h->launches += 1;
    h->last_n = n_per_iter;
    return collect_result(h, n_iter, out);
}

int rift_ile_av_info(const rift_ile_t *h, int32_t *level, int64_t *n_cells, int64_t *n_live, double *volume)
{
    if (!h)
        return RIFT_EINVAL;
    if (level)
        *level = h->av.level;
    if (n_cells)
        *n_cells = h->av.n_cells;
    if (n_live)
        *n_live = h->av.n_live;
    if (volume)
        *volume = h->av.V;
    return RIFT_OK;
}

}  // extern "C"
