// Likelihood kernels of the ILE hot path (arXiv:2505.11655 Sec. II A, Eq. (def:lnL:Decomposed),
// time-marginalised over a uniform grid as in the paper's timing appendix).
//
// This file holds the plain float64 path (one warp per sample, float64 throughout)
// and the per-sample coefficient kernel used for inspection.  The float32 tiled
// path is in k_tile.cu.
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
        double x = P.dist_marg ? 1.0 : P.d_ref / th[5];   // marginalised: terms at D = D_ref
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
            double v = P.dist_marg ? ln_dist_marg64(P, lin, quad) : lin - quad;
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

}  // namespace rift
