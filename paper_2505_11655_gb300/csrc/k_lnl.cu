// Likelihood kernels of the ILE hot path (arXiv:2505.11655 Sec. II A, Eq. (def:lnL:Decomposed),
// time-marginalised over a uniform grid as in the paper's timing appendix).
//
// Two implementations:
//   * lnl_fp64_kernel - the plain path: one warp per sample, float64 throughout.
//   * lnl_fp32_kernel - the fast path.  Samples arrive sorted by sky cell, so the
//     S = 64 samples of a tile need nearly the same Q window at every detector.  For
//     a chunk of time bins and one detector the tile forms, on the Q sample grid,
//         R[s, c] = sum_r C[s, r] Qr[r, iw0 + c],   r over the 2M real components
//     (C = (Re c_lm, Im c_lm), Qr = (Re Q_lm, Im Q_lm), so R = Re sum conj(c) Q),
//     a register-blocked 64 x W x 2M contraction from shared memory, then
//     interpolates R linearly at each bin's shifted time (interpolation commutes
//     with the mode sum), sums detectors, subtracts the template term and folds
//     the bins into a per-sample online log-sum-exp.
#include <cfloat>
#include <cmath>

#include "ile_kernels.h"

namespace rift {

// ======================================================================== shared pieces

template <typename T>
__device__ void sample_coeffs(const Problem &P, const double *th, Cx<T> *c /*[K*M]*/, double *dt /*[K]*/, T *x_out)
{
    Sky sky = sky_of(th[0], th[1], P.gmst);
    T s2p, c2p;
    sincos_t((T)(2.0 * th[2]), &s2p, &c2p);
    T cpow[kMaxPow + 1], spow[kMaxPow + 1];
    half_angle_powers<T>((T)th[4], cpow, spow);
    T x = (T)(P.d_ref / th[5]);
    for (int k = 0; k < P.K; ++k) {
        dt[k] = arrival_delay(P, k, sky);
        Cx<T> F = response<T>(P, k, sky, c2p, s2p);
        F.re *= x;
        F.im *= x;
        for (int m = 0; m < P.M; ++m)
            c[k * P.M + m] = cmul(F, harmonic<T>(P, m, cpow, spow, (T)th[3]));
    }
    if (x_out)
        *x_out = x;
}

// ======================================================================== FP64 plain path

constexpr int kF64Threads = 128;

__global__ void __launch_bounds__(kF64Threads) lnl_fp64_kernel(Problem P, const double *__restrict__ theta, int64_t n,
                                                               double *__restrict__ lnL_tmarg, double *__restrict__ lnL_t,
                                                               const double *__restrict__ lnpw, double *__restrict__ lnw,
                                                               int *err)
{
    extern __shared__ double2 sm64[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KM = P.K * P.M;
    double2 *cw = sm64 + warp * (KM + P.K + P.M);      // c[K*M], F[K], Y[M]
    double2 *Fw = cw + KM;
    double2 *Yw = Fw + P.K;
    __shared__ double dts[kF64Threads / 32][kMaxDet];
    const int wpb = blockDim.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * wpb + warp; s < n; s += (int64_t)gridDim.x * wpb) {
        const double *th = theta + 6 * s;
        Sky sky = sky_of(th[0], th[1], P.gmst);
        double x = P.d_ref / th[5];
        if (lane < P.K) {
            double s2p, c2p;
            sincos(2.0 * th[2], &s2p, &c2p);
            Cx<double> F = response<double>(P, lane, sky, c2p, s2p);
            Fw[lane] = make_double2(x * F.re, x * F.im);
            dts[warp][lane] = arrival_delay(P, lane, sky);
        }
        for (int m = lane; m < P.M; m += 32) {
            double cpow[kMaxPow + 1], spow[kMaxPow + 1];
            half_angle_powers<double>(th[4], cpow, spow);
            Cx<double> Y = harmonic<double>(P, m, cpow, spow, th[3]);
            Yw[m] = make_double2(Y.re, Y.im);
        }
        __syncwarp();
        for (int q = lane; q < KM; q += 32) {
            double2 F = Fw[q / P.M], Y = Yw[q % P.M];
            cw[q] = make_double2(F.x * Y.x - F.y * Y.y, F.x * Y.y + F.y * Y.x);
        }
        __syncwarp();
        // template term: kappa sum_k [ c^H U_k c + Re c^T V_k c ]
        double part = 0.0;
        for (int q = lane; q < KM; q += 32) {
            int k = q / P.M, a = q % P.M;
            const double2 *Ur = P.U64 + ((size_t)k * P.M + a) * P.M;
            const double2 *Vr = P.V64 + ((size_t)k * P.M + a) * P.M;
            double ur = 0, ui = 0, vr = 0, vi = 0;
            for (int b = 0; b < P.M; ++b) {
                double2 cb = cw[k * P.M + b], u = Ur[b], v = Vr[b];
                ur += u.x * cb.x - u.y * cb.y;
                ui += u.x * cb.y + u.y * cb.x;
                vr += v.x * cb.x - v.y * cb.y;
                vi += v.x * cb.y + v.y * cb.x;
            }
            double2 ca = cw[q];
            part += (ca.x * ur + ca.y * ui) + (ca.x * vr - ca.y * vi);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
            part += __shfl_xor_sync(0xffffffffu, part, o);
        const double quad = P.kappa * part;
        // data term per bin, online log-sum-exp per lane
        double mx = -INFINITY, sum = 0.0;
        for (int j = lane; j < P.n_t; j += 32) {
            double tj = P.t_lo + j * P.t_step;
            double lin = 0.0;
            for (int k = 0; k < P.K; ++k) {
                double u = (tj + dts[warp][k] - P.q_t0[k]) * P.fs;
                double fl = floor(u);
                if (!(fl >= 0.0) || fl + 1.0 > (double)(P.n_q - 1)) {
                    atomicOr(err, kErrRange);
                    continue;
                }
                int i = (int)fl;
                double f = u - fl;
                const double2 *Qk = P.Q64 + (size_t)k * P.M * P.n_q + i;
                for (int m = 0; m < P.M; ++m) {
                    double2 q0 = Qk[(size_t)m * P.n_q], q1 = Qk[(size_t)m * P.n_q + 1];
                    double2 c = cw[k * P.M + m];
                    double qr = (1.0 - f) * q0.x + f * q1.x;
                    double qi = (1.0 - f) * q0.y + f * q1.y;
                    lin += c.x * qr + c.y * qi;
                }
            }
            double v = lin - quad;
            if (lnL_t)
                lnL_t[s * P.n_t + j] = v;
            if (v > mx) {
                sum = sum * exp(mx - v) + 1.0;
                mx = v;
            } else {
                sum += exp(v - mx);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            double omx = __shfl_xor_sync(0xffffffffu, mx, o);
            double osum = __shfl_xor_sync(0xffffffffu, sum, o);
            double nm = fmax(mx, omx);
            double a = (mx == -INFINITY) ? 0.0 : sum * exp(mx - nm);
            double b = (omx == -INFINITY) ? 0.0 : osum * exp(omx - nm);
            mx = nm;
            sum = a + b;
        }
        if (lane == 0) {
            double r = mx + log(sum) - log((double)P.n_t);
            if (!isfinite(r))
                atomicOr(err, kErrNonFinite);
            lnL_tmarg[s] = r;
            if (lnw && lnpw)
                lnw[s] = r + lnpw[s];
        }
        __syncwarp();
    }
}

cudaError_t launch_lnl_fp64(const Problem &P, const double *theta, int64_t n, double *lnL_tmarg, double *lnL_t,
                            const double *lnpw, double *lnw, int *err, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = (size_t)(kF64Threads / 32) * (P.K * P.M + P.K + P.M) * sizeof(double2);
    int64_t want = (n + kF64Threads / 32 - 1) / (kF64Threads / 32);
    int grid = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    lnl_fp64_kernel<<<grid, kF64Threads, smem, st>>>(P, theta, n, lnL_tmarg, lnL_t, lnpw, lnw, err);
    return cudaGetLastError();
}

// ======================================================================== coefficients (inspection)

template <typename T>
__global__ void coeffs_kernel(Problem P, const double *__restrict__ theta, int64_t n, double2 *__restrict__ cout,
                              double *__restrict__ dtout, double *__restrict__ qout)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    Cx<T> c[kMaxDet * kMaxModes];
    double dt[kMaxDet];
    sample_coeffs<T>(P, theta + 6 * s, c, dt, (T *)nullptr);
    const int KM = P.K * P.M;
    if (cout)
        for (int q = 0; q < KM; ++q)
            cout[s * KM + q] = make_double2((double)c[q].re, (double)c[q].im);
    if (dtout)
        for (int k = 0; k < P.K; ++k)
            dtout[s * P.K + k] = dt[k];
    if (qout) {
        T tot = 0;
        for (int k = 0; k < P.K; ++k)
            for (int a = 0; a < P.M; ++a) {
                T ur = 0, ui = 0, vr = 0, vi = 0;
                for (int b = 0; b < P.M; ++b) {
                    size_t o = ((size_t)k * P.M + a) * P.M + b;
                    T uxr, uxi, vxr, vxi;
                    if (sizeof(T) == 8) {
                        uxr = (T)P.U64[o].x; uxi = (T)P.U64[o].y; vxr = (T)P.V64[o].x; vxi = (T)P.V64[o].y;
                    } else {
                        uxr = (T)P.U32[o].x; uxi = (T)P.U32[o].y; vxr = (T)P.V32[o].x; vxi = (T)P.V32[o].y;
                    }
                    Cx<T> cb = c[k * P.M + b];
                    ur += uxr * cb.re - uxi * cb.im;
                    ui += uxr * cb.im + uxi * cb.re;
                    vr += vxr * cb.re - vxi * cb.im;
                    vi += vxr * cb.im + vxi * cb.re;
                }
                Cx<T> ca = c[k * P.M + a];
                tot += (ca.re * ur + ca.im * ui) + (ca.re * vr - ca.im * vi);
            }
        qout[s] = (double)((T)P.kappa * tot);
    }
}

cudaError_t launch_coeffs(const Problem &P, bool fp64, const double *theta, int64_t n, double2 *c, double *dt,
                          double *quad, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    int grid = (int)((n + 127) / 128);
    if (fp64)
        coeffs_kernel<double><<<grid, 128, 0, st>>>(P, theta, n, c, dt, quad);
    else
        coeffs_kernel<float><<<grid, 128, 0, st>>>(P, theta, n, c, dt, quad);
    return cudaGetLastError();
}

// ======================================================================== FP32 tiled path

constexpr int kTS = 64;        // samples per tile
constexpr int kNCol = 256;     // largest Q window (columns) per chunk
constexpr int kColGroups = kNCol / 32;
constexpr int kTThreads = 256; // 8 warps
constexpr int kBinsPerLane = 5;  // bins per lane per chunk: a chunk holds <= 160 bins
constexpr int kMaxChunkBins = 32 * kBinsPerLane;

struct TileSmem {
    // byte offsets into dynamic shared memory
    size_t cs, buf, i0, f0, quad, end;
};

__host__ __device__ inline TileSmem tile_layout(int K, int M)
{
    TileSmem L;
    size_t o = 0;
    L.cs = o;
    o += (size_t)K * 2 * M * kTS * sizeof(float);
    L.buf = o;
    size_t qbytes = (size_t)2 * M * kNCol * sizeof(float);
    size_t rbytes = (size_t)kTS * kNCol * sizeof(float);
    o += qbytes > rbytes ? qbytes : rbytes;
    L.i0 = o;
    o += (size_t)K * kTS * sizeof(int);
    L.f0 = o;
    o += (size_t)K * kTS * sizeof(float);
    L.quad = o;
    o += (size_t)kTS * sizeof(float);
    L.end = (o + 15) & ~(size_t)15;
    return L;
}

size_t lnl_fp32_smem_bytes(const Problem &P) { return tile_layout(P.K, P.M).end; }

__global__ void __launch_bounds__(kTThreads, 1)
lnl_fp32_kernel(Problem P, BinTable bt, const double *__restrict__ theta, const uint32_t *__restrict__ perm, int64_t n,
                double *__restrict__ lnL_tmarg, double *__restrict__ lnL_t, const double *__restrict__ lnpw,
                double *__restrict__ lnw, int *err)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const TileSmem L = tile_layout(P.K, P.M);
    float *Cs = reinterpret_cast<float *>(smraw + L.cs);      // [K][2M][kTS]
    float *buf = reinterpret_cast<float *>(smraw + L.buf);    // Q chunk [2M][kNCol] or R [kTS][kNCol]
    int *i0s = reinterpret_cast<int *>(smraw + L.i0);         // [K][kTS]
    float *f0s = reinterpret_cast<float *>(smraw + L.f0);     // [K][kTS]
    float *qds = reinterpret_cast<float *>(smraw + L.quad);   // [kTS]
    __shared__ int lo_s[kMaxDet], hi_s[kMaxDet];
    __shared__ uint32_t gid_s[kTS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, M = P.M, R2 = 2 * M;
    const double beta = P.t_step * P.fs;
    const int64_t n_tiles = (n + kTS - 1) / kTS;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---------------- prologue: per-sample geometry, coefficients, template term
        if (tid < kMaxDet) {
            lo_s[tid] = INT_MAX;
            hi_s[tid] = INT_MIN;
        }
        __syncthreads();
        if (tid < kTS) {
            const int64_t si = tile * kTS + tid;
            uint32_t g = si < n ? perm[si] : 0xffffffffu;
            const bool valid = (int64_t)g < n;
            gid_s[tid] = valid ? g : 0xffffffffu;
            if (valid) {
                const double *th = theta + 6 * (int64_t)g;
                Cx<float> c[kMaxDet * kMaxModes];
                double dt[kMaxDet];
                sample_coeffs<float>(P, th, c, dt, (float *)nullptr);
                for (int k = 0; k < K; ++k) {
                    double u0 = (P.t_lo + dt[k] - P.q_t0[k]) * P.fs;
                    double fl = floor(u0);
                    int i0 = (int)fl;
                    i0s[k * kTS + tid] = i0;
                    f0s[k * kTS + tid] = (float)(u0 - fl);
                    atomicMin(&lo_s[k], i0);
                    atomicMax(&hi_s[k], i0);
                    for (int m = 0; m < M; ++m) {
                        Cs[(k * R2 + 2 * m) * kTS + tid] = c[k * M + m].re;
                        Cs[(k * R2 + 2 * m + 1) * kTS + tid] = c[k * M + m].im;
                    }
                }
            } else {
                for (int k = 0; k < K; ++k) {
                    i0s[k * kTS + tid] = 0;
                    f0s[k * kTS + tid] = 0.f;
                    for (int r = 0; r < R2; ++r)
                        Cs[(k * R2 + r) * kTS + tid] = 0.f;
                }
            }
        }
        __syncthreads();
        {
            // template term, 4 threads per sample, rows a = part, part + 4, ...
            const int s = tid >> 2, part = tid & 3;
            float acc = 0.f;
            for (int k = 0; k < K; ++k) {
                const float *Ck = Cs + (size_t)k * R2 * kTS;
                for (int a = part; a < M; a += 4) {
                    const float2 *Ur = P.U32 + ((size_t)k * M + a) * M;
                    const float2 *Vr = P.V32 + ((size_t)k * M + a) * M;
                    float ur = 0.f, ui = 0.f, vr = 0.f, vi = 0.f;
                    for (int b = 0; b < M; ++b) {
                        float cr = Ck[(2 * b) * kTS + s], ci = Ck[(2 * b + 1) * kTS + s];
                        float2 u = __ldg(Ur + b), v = __ldg(Vr + b);
                        ur = fmaf(u.x, cr, fmaf(-u.y, ci, ur));
                        ui = fmaf(u.x, ci, fmaf(u.y, cr, ui));
                        vr = fmaf(v.x, cr, fmaf(-v.y, ci, vr));
                        vi = fmaf(v.x, ci, fmaf(v.y, cr, vi));
                    }
                    float ar = Ck[(2 * a) * kTS + s], ai = Ck[(2 * a + 1) * kTS + s];
                    acc += (ar * ur + ai * ui) + (ar * vr - ai * vi);
                }
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (part == 0)
                qds[s] = (float)P.kappa * acc;
        }
        __syncthreads();

        int spread = 0;
        for (int k = 0; k < K; ++k)
            spread = max(spread, hi_s[k] - lo_s[k]);
        const bool direct = spread > kNCol - 16;   // pathological tile: no shared window
        // balanced chunking of the bins
        int jmax = (direct || !(beta > 0.0)) ? kMaxChunkBins : (int)floor((double)(kNCol - 8 - spread - 1) / beta) + 1;
        jmax = max(1, min(jmax, kMaxChunkBins));
        const int n_chunks = (P.n_t + jmax - 1) / jmax;
        const int jnom = (P.n_t + n_chunks - 1) / n_chunks;

        // per-warp running log-sum-exp for its 8 samples (s = warp + 8 p)
        float run_mx[8], run_sum[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            run_mx[p] = -INFINITY;
            run_sum[p] = 0.f;
        }

        for (int j0 = 0; j0 < P.n_t; j0 += jnom) {
            const int J = min(jnom, P.n_t - j0);
            float lin[8][kBinsPerLane];
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
                for (int q = 0; q < kBinsPerLane; ++q)
                    lin[p][q] = 0.f;

            for (int k = 0; k < K; ++k) {
                const float *Qk = P.Qr32 + (size_t)k * R2 * P.n_q_pad;
                const int *i0k = i0s + k * kTS;
                const float *f0k = f0s + k * kTS;
                if (!direct) {
                    const int base = lo_s[k] + __ldg(bt.bin_i + j0);
                    if (base < 0 && tid == 0)
                        atomicOr(err, kErrRange);
                    const int iw0 = max(base, 0) & ~3;
                    const int need = hi_s[k] + __ldg(bt.bin_i + j0 + J - 1) + 2 - iw0 + 1;
                    const int ncg = max(1, min(kColGroups, (need + 31) >> 5));
                    const int ncol4 = ncg * 8;   // float4 per row actually loaded
                    // stage the Q window of all 2M planes: buf[r][c] = Qr[r][iw0 + c]
                    for (int e = tid; e < R2 * ncol4; e += kTThreads) {
                        int r = e / ncol4, c4 = e - r * ncol4;
                        const float4 *src = reinterpret_cast<const float4 *>(Qk + (size_t)r * P.n_q_pad + iw0) + c4;
                        reinterpret_cast<float4 *>(buf + r * kNCol)[c4] = __ldg(src);
                    }
                    __syncthreads();
                    // register-blocked contraction: samples ty*8..+8, columns lane + 32 g
                    float acc[8][kColGroups];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int g = 0; g < kColGroups; ++g)
                            acc[i][g] = 0.f;
                    const float *Ck = Cs + (size_t)k * R2 * kTS + warp * 8;
#pragma unroll 2
                    for (int r = 0; r < R2; ++r) {
                        float4 a0 = *reinterpret_cast<const float4 *>(Ck + r * kTS);
                        float4 a1 = *reinterpret_cast<const float4 *>(Ck + r * kTS + 4);
                        float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                        float b[kColGroups];
#pragma unroll
                        for (int g = 0; g < kColGroups; ++g)
                            b[g] = (g < ncg) ? buf[r * kNCol + lane + 32 * g] : 0.f;
#pragma unroll
                        for (int i = 0; i < 8; ++i)
#pragma unroll
                            for (int g = 0; g < kColGroups; ++g)
                                acc[i][g] = fmaf(a[i], b[g], acc[i][g]);
                    }
                    __syncthreads();   // all reads of the Q window done: reuse buf for R
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int g = 0; g < kColGroups; ++g)
                            if (g < ncg)
                                buf[(warp * 8 + i) * kNCol + lane + 32 * g] = acc[i][g];
                    __syncthreads();
                    // interpolate R at each bin: warp -> samples warp + 8p, lane -> bins
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        const int s = warp + 8 * p;
                        const float *Rrow = buf + s * kNCol;
                        const int i0 = i0k[s] - iw0;
                        const float f0 = f0k[s];
                        const bool ok = gid_s[s] != 0xffffffffu;
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q) {
                            const int jj = lane + 32 * q;
                            if (ok && jj < J) {
                                const int j = j0 + jj;
                                float sf = f0 + __ldg(bt.bin_f + j);
                                int carry = sf >= 1.f;
                                float fr = sf - (float)carry;
                                int c = i0 + __ldg(bt.bin_i + j) + carry;
                                float r0 = Rrow[c], r1 = Rrow[c + 1];
                                lin[p][q] += fmaf(fr, r1 - r0, r0);
                            }
                        }
                    }
                    __syncthreads();   // R consumed before the next detector's Q window
                } else {
                    // direct evaluation from global memory (tiles without a shared window)
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        const int s = warp + 8 * p;
                        const int i0 = i0k[s];
                        const float f0 = f0k[s];
                        const bool ok = gid_s[s] != 0xffffffffu;
#pragma unroll
                        for (int q = 0; q < kBinsPerLane; ++q) {
                            const int jj = lane + 32 * q;
                            if (ok && jj < J) {
                                const int j = j0 + jj;
                                float sf = f0 + __ldg(bt.bin_f + j);
                                int carry = sf >= 1.f;
                                float fr = sf - (float)carry;
                                int c = i0 + __ldg(bt.bin_i + j) + carry;
                                if (c < 0 || c + 1 >= P.n_q) {
                                    atomicOr(err, kErrRange);
                                    continue;
                                }
                                float v = 0.f;
                                for (int r = 0; r < R2; ++r) {
                                    const float *row = Qk + (size_t)r * P.n_q_pad + c;
                                    float q0 = __ldg(row), q1 = __ldg(row + 1);
                                    v = fmaf(Cs[(k * R2 + r) * kTS + s], fmaf(fr, q1 - q0, q0), v);
                                }
                                lin[p][q] += v;
                            }
                        }
                    }
                }
            }
            // fold this chunk into the running log-sum-exp of each sample
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const int s = warp + 8 * p;
                const float qd = qds[s];
                const uint32_t g = gid_s[s];
                float cmx = -INFINITY;
#pragma unroll
                for (int q = 0; q < kBinsPerLane; ++q) {
                    const int jj = lane + 32 * q;
                    if (jj < J) {
                        lin[p][q] -= qd;
                        cmx = fmaxf(cmx, lin[p][q]);
                        if (lnL_t && g != 0xffffffffu)
                            lnL_t[(int64_t)g * P.n_t + j0 + jj] = (double)lin[p][q];
                    }
                }
#pragma unroll
                for (int o = 16; o; o >>= 1)
                    cmx = fmaxf(cmx, __shfl_xor_sync(0xffffffffu, cmx, o));
                const float nm = fmaxf(run_mx[p], cmx);
                float cs = 0.f;
#pragma unroll
                for (int q = 0; q < kBinsPerLane; ++q)
                    if (lane + 32 * q < J)
                        cs += __expf(lin[p][q] - nm);
#pragma unroll
                for (int o = 16; o; o >>= 1)
                    cs += __shfl_xor_sync(0xffffffffu, cs, o);
                run_sum[p] = (run_mx[p] == -INFINITY ? 0.f : run_sum[p] * __expf(run_mx[p] - nm)) + cs;
                run_mx[p] = nm;
            }
        }
        // epilogue
        if (lane < 8) {
            float mxv = run_mx[0], smv = run_sum[0];
#pragma unroll
            for (int p = 1; p < 8; ++p)
                if (lane == p) {
                    mxv = run_mx[p];
                    smv = run_sum[p];
                }
            const int s = warp + 8 * lane;
            const uint32_t g = gid_s[s];
            if (g != 0xffffffffu) {
                double r = (double)mxv + log((double)smv) - log((double)P.n_t);
                if (!isfinite(r))
                    atomicOr(err, kErrNonFinite);
                lnL_tmarg[g] = r;
                if (lnw && lnpw)
                    lnw[g] = r + lnpw[g];
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_lnl_fp32(const Problem &P, BinTable bt, const double *theta, const uint32_t *perm, int64_t n,
                            double *lnL_tmarg, double *lnL_t, const double *lnpw, double *lnw, int *err,
                            cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    size_t smem = lnl_fp32_smem_bytes(P);
    cudaError_t e = cudaFuncSetAttribute(lnl_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lnl_fp32_kernel, kTThreads, smem);
    if (per_sm < 1)
        per_sm = 1;
    int64_t tiles = (n + kTS - 1) / kTS;
    int64_t g = (int64_t)sms * per_sm;
    int grid = (int)(tiles < g ? tiles : g);
    lnl_fp32_kernel<<<grid, kTThreads, smem, st>>>(P, bt, theta, perm, n, lnL_tmarg, lnL_t, lnpw, lnw, err);
    return cudaGetLastError();
}

}  // namespace rift
