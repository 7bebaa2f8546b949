// Float64 re-evaluation of the samples that carry weight (precision mode RIFT_MIXED).
//
// At high signal-to-noise ratio ln L ~ 1e4 is a difference of data and template
// terms of the same size, and float32 rounding of those terms alone is ~1e-3
// (arXiv:2505.11655 Sec. II A, Eq. (def:lnL:Decomposed)).  Only samples whose weight
// can matter are redone: ln w_i >= max ln w - margin.  For each of them (one warp):
//   1. coefficients c_k,lm, arrival delays and the template term in float64;
//   2. the data term of every bin in float32 (float32 Q planes and coefficients),
//      which locates the bins that can matter for the time marginal;
//   3. every bin whose float32 ln L lies within kRefineBins of the sample's float32
//      maximum is recomputed in float64 (float64 Q, float64 interpolation);
//   4. the time marginal is a float64 log-sum-exp over the mixed values.
// Bins left in float32 sit more than kRefineBins below the maximum, where their
// absolute error (<~1e-2) cannot move the marginal by more than e^-kRefineBins.
#include <cfloat>
#include <cmath>

#include "ile_kernels.h"

namespace rift {

constexpr int kRefThreads = 128;   // 4 warps, one sample each
constexpr double kRefineBins = 40.0;

// Selection of the samples with key[i] >= max - margin, in ascending index order (so the
// list, and everything computed from it, is the same from run to run): block b of the
// grid owns the contiguous range [b per, (b + 1) per); pass 1 counts per block, a single
// block scans the counts, pass 2 writes each block's matches at its offset in order.
constexpr int kSelThreads = 256;
constexpr int kSelMaxBlocks = kSelectWords - 1;

__device__ __forceinline__ bool sel_take(const double *key, int64_t i, double cut) { return key[i] >= cut; }

__global__ void __launch_bounds__(kSelThreads) select_count_kernel(const double *__restrict__ key, int64_t n,
                                                                    const double *__restrict__ stats, int slot,
                                                                    double margin, uint32_t *__restrict__ blk)
{
    const double cut = stats[8 * slot + 4] - margin;   // max ln w (or max ln L) of the batch
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    uint32_t c = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kSelThreads)
        c += sel_take(key, i, cut) ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ uint32_t ws[kSelThreads / 32];
    if ((threadIdx.x & 31) == 0)
        ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kSelThreads / 32; ++w)
            t += ws[w];
        blk[blockIdx.x] = t;
    }
}

// exclusive scan of the nb block counts in place; the total goes to *count
__global__ void select_scan_kernel(uint32_t *__restrict__ blk, int nb, uint32_t *__restrict__ count)
{
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < nb; ++b) {
            const uint32_t c = blk[b];
            blk[b] = run;
            run += c;
        }
        *count = run;
    }
}

__global__ void __launch_bounds__(kSelThreads) select_write_kernel(const double *__restrict__ key, int64_t n,
                                                                    const double *__restrict__ stats, int slot,
                                                                    double margin, const uint32_t *__restrict__ blk,
                                                                    uint32_t *__restrict__ idx)
{
    const double cut = stats[8 * slot + 4] - margin;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    __shared__ uint32_t ws[kSelThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t base = blk[blockIdx.x];
    for (int64_t c0 = b0; c0 < b1; c0 += kSelThreads) {
        const int64_t i = c0 + threadIdx.x;
        const bool take = i < b1 && sel_take(key, i, cut);
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (lane == 0)
            ws[warp] = (uint32_t)__popc(mask);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) {
            before += w < warp ? ws[w] : 0u;
            total += ws[w];
        }
        if (take)
            idx[base + before + (uint32_t)__popc(mask & ((1u << lane) - 1))] = (uint32_t)i;
        base += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRefThreads) refine_kernel(Problem P, const double *__restrict__ theta,
                                                              const uint32_t *__restrict__ idx,
                                                              const uint32_t *__restrict__ count,
                                                              double *__restrict__ lnL_tmarg, const double *__restrict__ lnpw,
                                                              double *__restrict__ lnw, int *err,
                                                              const double *__restrict__ v32, int64_t v32_rows)
{
    extern __shared__ double rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int K = P.K, M = P.M, KM = K * M, NT = P.n_t;
    double2 *c64 = reinterpret_cast<double2 *>(rsm) + (size_t)warp * (KM + K + M);
    double2 *F64 = c64 + KM;
    double2 *Y64 = F64 + K;
    double *vals = rsm + (size_t)wpb * 2 * (KM + K + M) + (size_t)warp * NT;
    __shared__ double dts[kRefThreads / 32][kMaxDet];
    const uint32_t n_sel = *count;
    for (uint32_t w = blockIdx.x * wpb + warp; w < n_sel; w += gridDim.x * wpb) {
        const uint32_t s = idx[w];
        const double *th = theta + 6 * (size_t)s;
        Sky sky = sky_of(th[0], th[1], P.gmst);
        const double x = P.dist_marg ? 1.0 : P.d_ref / th[5];
        if (lane < K) {
            double s2p, c2p;
            sincos(2.0 * th[2], &s2p, &c2p);
            Cx<double> F = response<double>(P, lane, sky, c2p, s2p);
            F64[lane] = make_double2(x * F.re, x * F.im);
            dts[warp][lane] = arrival_delay(P, lane, sky);
        }
        for (int m = lane; m < M; m += 32) {
            double cpow[kMaxPow + 1], spow[kMaxPow + 1];
            half_angle_powers<double>(th[4], cpow, spow);
            Cx<double> Y = harmonic<double>(P, m, cpow, spow, th[3]);
            Y64[m] = make_double2(Y.re, Y.im);
        }
        __syncwarp();
        for (int q = lane; q < KM; q += 32) {
            const double2 F = F64[q / M], Y = Y64[q % M];
            c64[q] = make_double2(F.x * Y.x - F.y * Y.y, F.x * Y.y + F.y * Y.x);
        }
        __syncwarp();
        // template term in float64
        double part = 0.0;
        for (int q = lane; q < KM; q += 32) {
            const int k = q / M, a = q % M;
            const double2 *Ur = P.U64 + ((size_t)k * M + a) * M;
            const double2 *Vr = P.V64 + ((size_t)k * M + a) * M;
            double ur = 0, ui = 0, vr = 0, vi = 0;
#pragma unroll 7
            for (int b = 0; b < M; ++b) {
                const double2 cb = c64[k * M + b], u = Ur[b], v = Vr[b];
                ur += u.x * cb.x - u.y * cb.y;
                ui += u.x * cb.y + u.y * cb.x;
                vr += v.x * cb.x - v.y * cb.y;
                vi += v.x * cb.y + v.y * cb.x;
            }
            const double2 ca = c64[q];
            part += (ca.x * ur + ca.y * ui) + (ca.x * vr - ca.y * vi);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            part += __shfl_xor_sync(0xffffffffu, part, o);
        const double quad = P.kappa * part;
        // float32 ln L at every bin: from the tiled kernel's second pass over the selected
        // samples when it ran for this one, else recomputed here
        float mx32 = -INFINITY;
        if ((int64_t)w < v32_rows) {
            const double *row = v32 + (size_t)w * NT;
            for (int j = lane; j < NT; j += 32) {
                const double v = row[j];
                vals[j] = v;
                mx32 = fmaxf(mx32, (float)v);
            }
        } else
        for (int j = lane; j < NT; j += 32) {
            const double tj = P.t_lo + j * P.t_step;
            float lin = 0.f;
            for (int k = 0; k < K; ++k) {
                const double u = (tj + dts[warp][k] - P.q_t0[k]) * P.fs;
                const double fl = floor(u);
                if (!(fl >= 0.0) || fl + 1.0 > (double)(P.n_q - 1)) {
                    atomicOr(err, kErrRange);
                    continue;
                }
                const int i = (int)fl;
                const float f = (float)(u - fl);
                const float *Qk = P.Qr32 + (size_t)k * 2 * M * P.n_q_pad + i;
                // the loads of several modes in flight at once (the Q planes live in L2)
#pragma unroll 7
                for (int m = 0; m < M; ++m) {
                    const double2 c = c64[k * M + m];
                    const float *qr = Qk + (size_t)(2 * m) * P.n_q_pad, *qi = qr + P.n_q_pad;
                    const float vr = fmaf(f, qr[1] - qr[0], qr[0]), vi = fmaf(f, qi[1] - qi[0], qi[0]);
                    lin = fmaf((float)c.x, vr, fmaf((float)c.y, vi, lin));
                }
            }
            const double v = P.dist_marg ? (double)ln_dist_marg32(P, lin, (float)quad) : (double)lin - quad;
            vals[j] = v;
            mx32 = fmaxf(mx32, (float)v);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            mx32 = fmaxf(mx32, __shfl_xor_sync(0xffffffffu, mx32, o));
        __syncwarp();
        // float64 data term at the bins that can matter
        double mx = -INFINITY;
        for (int j = lane; j < NT; j += 32) {
            double v = vals[j];
            if (v >= (double)mx32 - kRefineBins) {
                const double tj = P.t_lo + j * P.t_step;
                double lin = 0.0;
                for (int k = 0; k < K; ++k) {
                    const double u = (tj + dts[warp][k] - P.q_t0[k]) * P.fs;
                    const double fl = floor(u);
                    if (!(fl >= 0.0) || fl + 1.0 > (double)(P.n_q - 1))
                        continue;
                    const int i = (int)fl;
                    const double f = u - fl;
                    const double2 *Qk = P.Q64 + (size_t)k * M * P.n_q + i;
#pragma unroll 7
                    for (int m = 0; m < M; ++m) {
                        const double2 q0 = Qk[(size_t)m * P.n_q], q1 = Qk[(size_t)m * P.n_q + 1];
                        const double2 c = c64[k * M + m];
                        lin += c.x * ((1.0 - f) * q0.x + f * q1.x) + c.y * ((1.0 - f) * q0.y + f * q1.y);
                    }
                }
                v = P.dist_marg ? ln_dist_marg64(P, lin, quad) : lin - quad;
                vals[j] = v;
            }
            mx = fmax(mx, v);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        double sum = 0.0;
        for (int j = lane; j < NT; j += 32)
            sum += exp(vals[j] - mx);
#pragma unroll
        for (int o = 16; o; o >>= 1)
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            const double r = mx + log(sum) - log((double)NT);
            if (!isfinite(r))
                atomicOr(err, kErrNonFinite);
            lnL_tmarg[s] = r;
            if (lnw && lnpw)
                lnw[s] = r + lnpw[s];
        }
        __syncwarp();
    }
}

cudaError_t launch_select(const double *key, int64_t n, const double *stats, int slot, double margin, uint32_t *idx,
                          uint32_t *count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    // block counts live after the count word
    uint32_t *blk = count + 1;
    const int64_t want = (n + 4 * kSelThreads - 1) / (4 * kSelThreads);
    const int grid = (int)(want < kSelMaxBlocks ? (want > 0 ? want : 1) : kSelMaxBlocks);
    select_count_kernel<<<grid, kSelThreads, 0, st>>>(key, n, stats, slot, margin, blk);
    select_scan_kernel<<<1, 32, 0, st>>>(blk, grid, count);
    select_write_kernel<<<grid, kSelThreads, 0, st>>>(key, n, stats, slot, margin, blk, idx);
    return cudaGetLastError();
}

cudaError_t launch_refine(const Problem &P, const double *theta, const uint32_t *idx, const uint32_t *count,
                          int64_t max_count, double *lnL_tmarg, const double *lnpw, double *lnw, int *err,
                          cudaStream_t st, const double *v32, int64_t v32_rows)
{
    if (max_count <= 0)
        return cudaSuccess;
    const int wpb = kRefThreads / 32;
    const size_t smem = sizeof(double) * ((size_t)wpb * 2 * (P.K * P.M + P.K + P.M) + (size_t)wpb * P.n_t);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem(refine_kernel);
        if (e != cudaSuccess)
            return e;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (max_count + wpb - 1) / wpb;
    const int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    refine_kernel<<<grid, kRefThreads, smem, st>>>(P, theta, idx, count, lnL_tmarg, lnpw, lnw, err, v32,
                                                   v32 ? v32_rows : 0);
    return cudaGetLastError();
}

cudaError_t prepare_refine_kernels()
{
    return allow_max_dynamic_smem(refine_kernel);
}

}  // namespace rift
