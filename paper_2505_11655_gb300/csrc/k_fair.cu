// Fair draws from a batch of weighted samples: the final ILE pass (arXiv:2505.11655,
// Sec. II, the closing paragraph of the method overview; Sec. II D's two-step fair draw
// from weighted samples).  A sample i is drawn, with replacement, with probability
// w_i / sum w; its time bin j with probability exp(ln L_ij) / sum_j exp(ln L_ij) (the
// time prior is uniform on the grid).
//
// Every choice is made exactly in integer arithmetic, so that it does not depend on
// summation order: item weights are W_i = floor(exp(x_i - max x) 2^S) with
// S = 62 - ceil(log2 n) (0 for non-finite x_i); draw d takes the 53-bit integers U of
// Philox4x32-10 under key = seed, counter = (d low, d high, 0xFFFFFFFF, 0) (words 0,1
// for the sample, 2,3 for the time bin) and chooses the first item whose running sum of
// W exceeds floor(U Total / 2^53).
#include <cfloat>
#include <cmath>

#include "ile_kernels.h"

namespace rift {

__device__ __forceinline__ uint64_t fix_weight(double x, double mx, int S)
{
    if (!isfinite(x))
        return 0ull;
    return (uint64_t)ldexp(exp(x - mx), S);
}

__device__ __forceinline__ uint64_t u53_int(uint32_t a, uint32_t b)
{
    return ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
}

// floor(U tot / 2^53) for U < 2^53, tot < 2^63
__device__ __forceinline__ uint64_t fix_threshold(uint64_t U, uint64_t tot)
{
    const uint64_t lo = U * tot, hi = __umul64hi(U, tot);
    return (hi << 11) | (lo >> 53);
}

__global__ void fair_weights_kernel(const double *__restrict__ lnw, int64_t n, const double *__restrict__ stats,
                                    int slot, int S, uint64_t *__restrict__ W, uint64_t *__restrict__ E)
{
    const double mx = stats[8 * slot + 4];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t w = fix_weight(lnw[i], mx, S);
        W[i] = w;
        E[i] = w;   // scanned in place to exclusive running sums
    }
}

// One thread per draw: binary search for the first i with E[i] + W[i] > T.
__global__ void fair_select_kernel(const uint64_t *__restrict__ W, const uint64_t *__restrict__ E, int64_t n,
                                   uint64_t seed, int64_t n_draws, const double *__restrict__ theta,
                                   int64_t *__restrict__ idx, double *__restrict__ theta_sel,
                                   uint64_t *__restrict__ U_time)
{
    const uint64_t tot = E[n - 1] + W[n - 1];
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_draws;
         d += (int64_t)gridDim.x * blockDim.x) {
        const U4 r = philox10(U4{(uint32_t)(uint64_t)d, (uint32_t)((uint64_t)d >> 32), 0xFFFFFFFFu, 0u}, k0, k1);
        const uint64_t T = fix_threshold(u53_int(r.x, r.y), tot);
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (E[mid] + W[mid] > T)
                hi = mid;
            else
                lo = mid + 1;
        }
        idx[d] = lo;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            theta_sel[6 * d + c] = theta[6 * lo + c];
        U_time[d] = u53_int(r.z, r.w);
    }
}

// One warp per draw: the time bin from the draw's per-bin ln L (row of n_t values).
__global__ void fair_time_kernel(const double *__restrict__ lnL_t, int64_t m, int n_t, int S2,
                                 const uint64_t *__restrict__ U_time, double t_lo, double t_step,
                                 int32_t *__restrict__ j_out, double *__restrict__ t_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < m; d += warps) {
        const double *row = lnL_t + (size_t)d * n_t;
        double mx = -INFINITY;
        for (int j = lane; j < n_t; j += 32)
            if (isfinite(row[j]))
                mx = fmax(mx, row[j]);
#pragma unroll
        for (int o = 16; o; o >>= 1)
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        uint64_t tot = 0;
        for (int j = lane; j < n_t; j += 32)
            tot += fix_weight(row[j], mx, S2);
#pragma unroll
        for (int o = 16; o; o >>= 1)
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        int chosen = n_t - 1;
        if (tot > 0) {
            const uint64_t T = fix_threshold(U_time[d], tot);
            uint64_t base = 0;
            for (int j0 = 0; j0 < n_t; j0 += 32) {
                const int j = j0 + lane;
                const uint64_t w = j < n_t ? fix_weight(row[j], mx, S2) : 0ull;
                uint64_t inc = w;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o)
                        inc += y;
                }
                const unsigned hit = __ballot_sync(0xffffffffu, j < n_t && base + inc > T);
                if (hit) {
                    chosen = j0 + __ffs(hit) - 1;
                    break;
                }
                base += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        if (lane == 0) {
            j_out[d] = chosen;
            t_out[d] = t_lo + chosen * t_step;
        }
    }
}

static int fix_shift(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n)
        ++c;
    return 62 - c;
}

static int blocks_for(int64_t n, int threads)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

cudaError_t launch_fair_select(const double *lnw, int64_t n, const double *stats, int slot, uint64_t *W,
                               uint64_t *E, uint64_t *scan_scratch, uint64_t seed, int64_t n_draws,
                               const double *theta, int64_t *idx, double *theta_sel, uint64_t *U_time,
                               cudaStream_t st, int *launched)
{
    int k = 0;
    fair_weights_kernel<<<blocks_for(n, 256), 256, 0, st>>>(lnw, n, stats, slot, fix_shift(n), W, E);
    cudaError_t e = launch_scan_u64(E, n, scan_scratch, st, &k);
    if (e != cudaSuccess)
        return e;
    fair_select_kernel<<<blocks_for(n_draws, 128), 128, 0, st>>>(W, E, n, seed, n_draws, theta, idx, theta_sel,
                                                                  U_time);
    if (launched)
        *launched = k + 2;
    return cudaGetLastError();
}

cudaError_t launch_fair_time(const double *lnL_t, int64_t m, int n_t, const uint64_t *U_time, double t_lo,
                             double t_step, int32_t *j_out, double *t_out, cudaStream_t st)
{
    if (m <= 0)
        return cudaSuccess;
    fair_time_kernel<<<blocks_for(m * 32, 256), 256, 0, st>>>(lnL_t, m, n_t, fix_shift(n_t), U_time, t_lo, t_step,
                                                              j_out, t_out);
    return cudaGetLastError();
}

}  // namespace rift
