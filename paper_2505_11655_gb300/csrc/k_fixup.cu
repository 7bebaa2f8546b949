// Large-term correction of the float32 likelihood path.
//
// ln L_j = lin_j - quad is the difference of the data term and the template term of
// arXiv:2505.11655 Eq. (def:lnL:Decomposed).  For a sample near the lower distance bound
// both terms reach 1e3..1e4 while their difference is a large negative number, and float32
// rounding of the coefficients c_k,lm = (D_ref/D) F_k Y_lm and of the template term moves
// ln L by ~3e-7 (|lnL| + 2 quad): up to ~1e-2.  Nearly all of that error is common to
// every time bin of the sample (the template term, and the scale of the coefficients), so
// it is removed per sample rather than per bin:
//
//   1. the float32 kernel writes, beside ln L_tmarg = LSE_j(lin_j) - quad32 - ln n_t (the
//      difference taken in float64), the float32 template term quad32, the largest float32
//      data term m32 and a block of bins holding the bin of m32;
//   2. samples with quad32 + |m32| above a threshold (the float32 error can exceed the
//      parity bar there) are listed;
//   3. for each listed sample, with the coefficients from float64 geometry:
//        the template term in double-float (~44 bits), written through the symmetry of
//        U (Hermitian) and V (symmetric) and the form Y_lm = d_lm(iota) exp(-i m phi):
//          c^H U_k c = |s_k|^2 sum_D exp(i D phi) G_k,D,  G_k,D = sum_{m_a - m_b = D} d_a d_b U_k,ab
//          c^T V_k c = s_k^2  sum_S exp(-i S phi) H_k,S,  H_k,S = sum_{m_a + m_b = S} d_a d_b V_k,ab
//        with s_k = (D_ref/D) F_k;
//        the bin of the block with the largest data term (a float32 search when the block
//        holds several bins), and the data term there in double-float, from a double-float
//        copy of Q;
//      and ln L_tmarg moves by (quad32 - quad) + (lin(j*) - m32): the error of the float32
//      data term is the same at every bin near the maximum (a scale error of the
//      coefficients), and the bins far below it do not move the log-sum-exp.
// The per-bin values (when requested) move by the same amount.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "df.cuh"
#include "ile_kernels.h"

namespace rift {

constexpr int kFixMaxWarps = 16;   // warps per block: as many as the shared memory holds, up to this

// --------------------------------------------------------------- double-float copies

__global__ void fix_prep_kernel(const double2 *__restrict__ U64, const double2 *__restrict__ V64,
                                const double2 *__restrict__ Q64, int K, int M, int n_q, FixTables T, float4 *ua,
                                float4 *vb, float4 *qdf)
{
    const int64_t nua = (int64_t)K * T.nA, nvb = (int64_t)K * T.nB, nq = (int64_t)K * M * n_q;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nua + nvb + nq;
         e += (int64_t)gridDim.x * blockDim.x) {
        double2 v;
        float4 *dst;
        if (e < nua) {
            const int k = (int)(e / T.nA), p = (int)(e - (int64_t)k * T.nA);
            const int i = T.a_ij[p] & 255, j = T.a_ij[p] >> 8;
            v = U64[((size_t)k * M + i) * M + j];
            dst = ua + e;
        } else if (e < nua + nvb) {
            const int64_t f = e - nua;
            const int k = (int)(f / T.nB), p = (int)(f - (int64_t)k * T.nB);
            const int i = T.b_ij[p] & 255, j = T.b_ij[p] >> 8;
            v = V64[((size_t)k * M + i) * M + j];
            if (i != j)
                v = make_double2(2.0 * v.x, 2.0 * v.y);   // the pair (j, i) of the symmetric V
            dst = vb + f;
        } else {
            const int64_t f = e - nua - nvb;
            v = Q64[f];
            dst = qdf + f;
        }
        const df re = df_of(v.x), im = df_of(v.y);
        *dst = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

// --------------------------------------------------------------- selection

__global__ void fix_select_kernel(const float *__restrict__ aq, const float *__restrict__ am, int64_t n, float thr,
                                  uint32_t *__restrict__ idx, uint32_t *__restrict__ count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    if (i < n)
        take = aq[i] + fabsf(am[i]) > thr;   // a non-finite value is flagged by the kernel that wrote it
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    if (!mask)
        return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader)
        base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (take)
        idx[base + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)i;
}

// --------------------------------------------------------------- correction

// Per-warp shared memory: float64 rows [K + 1][32] (the Q position u0_k of the first bin,
// then the template term), float rows [nf][32] (double-float s_k, d_lm, exp(-i n phi)), and
// [32] the bin at which each sample's data term is evaluated.
__host__ __device__ inline int fix_float_rows(int K, int M, int dmax) { return 4 * K + 2 * M + 4 * (dmax + 1); }

__host__ __device__ inline size_t fix_warp_bytes(int K, int M, int dmax)
{
    return (size_t)(K + 1) * 32 * 8 + (size_t)fix_float_rows(K, M, dmax) * 32 * 4 + 32 * 4;
}

__global__ void __launch_bounds__(32 * kFixMaxWarps)
fix_kernel(Problem P, BinTable bt, FixTables T, const double *__restrict__ theta, const uint32_t *__restrict__ idx,
           const uint32_t *__restrict__ count, PeakOut po, int blen, double *__restrict__ lnL_tmarg,
           double *__restrict__ lnL_t, const double *__restrict__ lnpw, double *__restrict__ lnw, int *err)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = P.K, M = P.M, NT = P.n_t;
    const int nph = T.dmax + 1;
    unsigned char *wb = fsm + fix_warp_bytes(K, M, T.dmax) * warp;
    double *rd = reinterpret_cast<double *>(wb);                 // [K + 1][32]
    float *rf = reinterpret_cast<float *>(rd + (K + 1) * 32);     // [nf][32]
    float *c32 = rf + fix_float_rows(K, M, T.dmax) * 32;
    // rows of rf: s_k (re.hi, re.lo, im.hi, im.lo) at 4k; d_lm (hi, lo) at 4K + 2m;
    // exp(-i n phi) (re.hi, re.lo, im.hi, im.lo) at 4K + 2M + 4n
    const int rs = 0, rdl = 4 * K, rph = 4 * K + 2 * M;
    const double beta = P.t_step * P.fs;
    const uint32_t cnt = *count;
    const int nw = (int)(blockDim.x >> 5);
    // batch b of 32 listed samples goes to block b % gridDim.x, warp b / gridDim.x (round
    // robin over the blocks first, so that a short list still spreads over every SM)
    if ((int64_t)blockIdx.x * 32 >= (int64_t)cnt)
        return;   // no listed sample for this block (the grid is sized for every sample)
    // the pair tables and the double-float U, V of every detector, staged once per block
    float4 *sua = reinterpret_cast<float4 *>(fsm + fix_warp_bytes(K, M, T.dmax) * nw);
    float4 *svb = sua + K * T.nA;
    uint16_t *saij = reinterpret_cast<uint16_t *>(svb + K * T.nB);
    uint16_t *sbij = saij + T.nA;
    for (int e = threadIdx.x; e < K * T.nA; e += blockDim.x)
        sua[e] = T.ua[e];
    for (int e = threadIdx.x; e < K * T.nB; e += blockDim.x)
        svb[e] = T.vb[e];
    for (int e = threadIdx.x; e < T.nA; e += blockDim.x)
        saij[e] = T.a_ij[e];
    for (int e = threadIdx.x; e < T.nB; e += blockDim.x)
        sbij[e] = T.b_ij[e];
    __syncthreads();
    // this lane's sample: the double-float value at rows (row, row + 1)
    auto ld = [&](int row) { return df{rf[row * 32 + lane], rf[(row + 1) * 32 + lane]}; };

    for (int64_t base = ((int64_t)warp * gridDim.x + blockIdx.x) * 32; base < (int64_t)cnt;
         base += (int64_t)gridDim.x * nw * 32) {
        const int64_t e = base + lane;
        const bool active = e < (int64_t)cnt;
        const uint32_t g = active ? idx[e] : 0u;

        // ---- phase A, one sample per lane: geometry in float64, rounded to double-float
        {
            double th[6] = {0.0, 0.0, 0.0, 0.0, 0.0, P.d_ref};   // inert values on idle lanes
            if (active)
                for (int d = 0; d < 6; ++d)
                    th[d] = theta[6 * (int64_t)g + d];
            const Sky sky = sky_of(th[0], th[1], P.gmst);
            const double n0 = sky.cd * sky.ch, n1 = sky.cd * sky.sh, n2 = sky.sd;
            double s2p, c2p;
            sincos(2.0 * th[2], &s2p, &c2p);
            const double x = P.d_ref / th[5];
            for (int k = 0; k < K; ++k) {
                rd[k * 32 + lane] = fma(P.xfs[k][0], n0, fma(P.xfs[k][1], n1, fma(P.xfs[k][2], n2, P.ufs0[k])));
                const Cx<double> F = response<double>(P, k, sky, c2p, s2p);
                const df sr = df_of(x * F.re), si = df_of(x * F.im);
                rf[(rs + 4 * k) * 32 + lane] = sr.hi;
                rf[(rs + 4 * k + 1) * 32 + lane] = sr.lo;
                rf[(rs + 4 * k + 2) * 32 + lane] = si.hi;
                rf[(rs + 4 * k + 3) * 32 + lane] = si.lo;
            }
            double cpow[kMaxPow + 1], spow[kMaxPow + 1];
            half_angle_powers<double>(th[4], cpow, spow);
            for (int m = 0; m < M; ++m) {
                double d = 0.0;
                for (int t = 0; t < P.wn[m]; ++t)
                    d += P.wcoef[m][t] * cpow[P.wpc[m][t]] * spow[P.wps[m][t]];
                const df dd = df_of(d);
                rf[(rdl + 2 * m) * 32 + lane] = dd.hi;
                rf[(rdl + 2 * m + 1) * 32 + lane] = dd.lo;
            }
            double sp, cp;
            sincos(th[3], &sp, &cp);
            double er = 1.0, ei = 0.0;   // exp(-i n phi), n = 0, 1, ...
            for (int nn = 0; nn < nph; ++nn) {
                const df a = df_of(er), b = df_of(ei);
                rf[(rph + 4 * nn) * 32 + lane] = a.hi;
                rf[(rph + 4 * nn + 1) * 32 + lane] = a.lo;
                rf[(rph + 4 * nn + 2) * 32 + lane] = b.hi;
                rf[(rph + 4 * nn + 3) * 32 + lane] = b.lo;
                const double t = er * cp + ei * sp;
                ei = ei * cp - er * sp;
                er = t;
            }
        }
        __syncwarp();

        // ---- the template term in double-float, one sample per lane
        {
            df A[kMaxDet];
            dfc B[kMaxDet];
#pragma unroll
            for (int k = 0; k < kMaxDet; ++k) {
                A[k] = {0.f, 0.f};
                B[k] = {{0.f, 0.f}, {0.f, 0.f}};
            }
            for (int D = 0; D <= T.dmax; ++D) {
                dfc G[kMaxDet];
#pragma unroll
                for (int k = 0; k < kMaxDet; ++k)
                    G[k] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 2
                for (int p = T.a_start[D]; p < T.a_start[D + 1]; ++p) {
                    const int ij = saij[p];
                    const df w = df_mul(ld(rdl + 2 * (ij & 255)), ld(rdl + 2 * (ij >> 8)));
#pragma unroll
                    for (int k = 0; k < kMaxDet; ++k)
                        if (k < K) {
                            const float4 u = sua[k * T.nA + p];
                            df_acc(G[k].re, w, {u.x, u.y});
                            df_acc(G[k].im, w, {u.z, u.w});
                        }
                }
#pragma unroll
                for (int k = 0; k < kMaxDet; ++k)
                    G[k] = {df_norm(G[k].re), df_norm(G[k].im)};
                // A_k += G_0, or 2 Re(exp(i D phi) G_D) = 2 (Re e Re G + Im e Im G), e = exp(-i D phi)
                const df er = ld(rph + 4 * D), ei = ld(rph + 4 * D + 2);
#pragma unroll
                for (int k = 0; k < kMaxDet; ++k)
                    if (k < K) {
                        if (D == 0) {
                            A[k] = df_add(A[k], G[k].re);
                        } else {
                            const df t = df_add(df_mul(er, G[k].re), df_mul(ei, G[k].im));
                            A[k] = df_add(A[k], df_add(t, t));
                        }
                    }
            }
            for (int S = -T.dmax; S <= T.dmax; ++S) {
                dfc H[kMaxDet];
#pragma unroll
                for (int k = 0; k < kMaxDet; ++k)
                    H[k] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 2
                for (int p = T.b_start[S + T.dmax]; p < T.b_start[S + T.dmax + 1]; ++p) {
                    const int ij = sbij[p];
                    const df w = df_mul(ld(rdl + 2 * (ij & 255)), ld(rdl + 2 * (ij >> 8)));
#pragma unroll
                    for (int k = 0; k < kMaxDet; ++k)
                        if (k < K) {
                            const float4 v = svb[k * T.nB + p];
                            df_acc(H[k].re, w, {v.x, v.y});
                            df_acc(H[k].im, w, {v.z, v.w});
                        }
                }
#pragma unroll
                for (int k = 0; k < kMaxDet; ++k)
                    H[k] = {df_norm(H[k].re), df_norm(H[k].im)};
                // exp(-i S phi): the table entry for S >= 0, its conjugate for S < 0
                const int a = S < 0 ? -S : S;
                dfc e{ld(rph + 4 * a), ld(rph + 4 * a + 2)};
                if (S < 0)
                    e.im = {-e.im.hi, -e.im.lo};
#pragma unroll
                for (int k = 0; k < kMaxDet; ++k)
                    if (k < K) {
                        const dfc t = dfc_mul(e, H[k]);
                        B[k].re = df_add(B[k].re, t.re);
                        B[k].im = df_add(B[k].im, t.im);
                    }
            }
            // quad = kappa sum_k |s_k|^2 A_k + Re(s_k^2 B_k)
            df q = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < kMaxDet; ++k)
                if (k < K) {
                    const df sr = ld(rs + 4 * k), si = ld(rs + 4 * k + 2);
                    const df rr = df_mul(sr, sr), ii = df_mul(si, si), ri = df_mul(sr, si);
                    const df abs2 = df_add(rr, ii), s2r = df_sub(rr, ii), s2i = df_add(ri, ri);
                    q = df_add(q, df_mul(abs2, A[k]));
                    q = df_add(q, df_sub(df_mul(s2r, B[k].re), df_mul(s2i, B[k].im)));
                }
            rd[K * 32 + lane] = P.kappa * df_to_double(q);
        }
        __syncwarp();

        // ---- phase B: the bin of the largest data term in the kernel's block (float32
        // search; lanes = (sample, bin of the block) pairs), then the data term there in
        // double-float, one sample per lane
        const int nb = (int)((int64_t)cnt - base < 32 ? (int64_t)cnt - base : 32);
        int *jbest = reinterpret_cast<int *>(c32);   // [32] the bin each sample is evaluated at
        if (blen <= 1) {
            if (lane < nb)
                jbest[lane] = po.j[g];
        } else {
            int lps = 1;   // lanes per sample: the block length rounded up to a power of two
            while (lps < blen)
                lps <<= 1;
            const int spr = 32 / lps;   // samples per round
            for (int r0 = 0; r0 < nb; r0 += spr) {
                const int t = r0 + lane / lps, b = lane % lps;
                const uint32_t gt = __shfl_sync(0xffffffffu, g, t & 31);
                float best = -INFINITY;
                int bj = INT_MAX;
                if (t < nb && b < blen) {
                    const int jb = po.j[gt], j = jb + b;
                    if (jb >= 0 && j < NT) {
                        float lin = 0.f;
                        bool ok = true;
                        for (int k = 0; k < K && ok; ++k) {
                            const double u0 = rd[k * 32 + t];
                            const double fl = floor(u0);
                            const float sf = (float)(u0 - fl) + bt.bin_f[j];
                            const int carry = sf >= 1.f;
                            const float fr = sf - (float)carry;
                            const int c = (int)fl + bt.bin_i[j] + carry;
                            if (c < 0 || c + 1 >= P.n_q) {
                                ok = false;
                                break;
                            }
                            const float sr = rf[(rs + 4 * k) * 32 + t], si = rf[(rs + 4 * k + 2) * 32 + t];
                            const float *Qk = P.Qr32 + (size_t)k * 2 * M * P.n_q_pad + c;
#pragma unroll 7
                            for (int m = 0; m < M; ++m) {
                                const int mm = P.mode_m[m], a = mm < 0 ? -mm : mm;
                                const float d = rf[(rdl + 2 * m) * 32 + t];
                                const float er = rf[(rph + 4 * a) * 32 + t];
                                const float ei = mm < 0 ? -rf[(rph + 4 * a + 2) * 32 + t] : rf[(rph + 4 * a + 2) * 32 + t];
                                const float yr = d * er, yi = d * ei;
                                const float cr = sr * yr - si * yi, ci = sr * yi + si * yr;
                                const float *qr = Qk + (size_t)(2 * m) * P.n_q_pad, *qi = qr + P.n_q_pad;
                                const float vr = fmaf(fr, qr[1] - qr[0], qr[0]), vi = fmaf(fr, qi[1] - qi[0], qi[0]);
                                lin = fmaf(cr, vr, fmaf(ci, vi, lin));
                            }
                        }
                        if (ok) {
                            best = lin;
                            bj = j;
                        }
                    }
                }
                // the largest value of the sample's bins, the lowest bin among equals
                for (int o = 1; o < lps; o <<= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                    if (ov > best || (ov == best && oj < bj)) {
                        best = ov;
                        bj = oj;
                    }
                }
                if (b == 0 && t < nb)
                    jbest[t] = bj;
            }
        }
        __syncwarp();
        double corr = 0.0;
        bool good = false;
        if (lane < nb) {
            const int j = jbest[lane];
            if (j != INT_MAX) {
                df acc = {0.f, 0.f};
                good = true;
                for (int k = 0; k < K; ++k) {
                    const double u = rd[k * 32 + lane] + (double)j * beta;
                    const double fl = floor(u);
                    if (!(fl >= 0.0) || fl + 1.0 > (double)(P.n_q - 1)) {
                        good = false;
                        break;
                    }
                    const int i = (int)fl;
                    const df f = df_of(u - fl);
                    const dfc sk{ld(rs + 4 * k), ld(rs + 4 * k + 2)};
                    const float4 *qk = T.qdf + (size_t)k * M * P.n_q + i;
                    for (int m = 0; m < M; ++m) {
                        const float4 q0 = qk[(size_t)m * P.n_q], q1 = qk[(size_t)m * P.n_q + 1];
                        const df r0{q0.x, q0.y}, r1{q1.x, q1.y}, i0{q0.z, q0.w}, i1{q1.z, q1.w};
                        const df qre = df_add(r0, df_mul(f, df_sub(r1, r0)));
                        const df qim = df_add(i0, df_mul(f, df_sub(i1, i0)));
                        // Y_lm = d_lm exp(-i m phi): the table entry for m >= 0, its conjugate for m < 0
                        const int mm = P.mode_m[m], a = mm < 0 ? -mm : mm;
                        const df d = ld(rdl + 2 * m);
                        df er = ld(rph + 4 * a), ei = ld(rph + 4 * a + 2);
                        if (mm < 0)
                            ei = {-ei.hi, -ei.lo};
                        const dfc c = dfc_mul(sk, dfc{df_mul(d, er), df_mul(d, ei)});
                        acc = df_add(acc, df_add(df_mul(c.re, qre), df_mul(c.im, qim)));
                    }
                }
                if (good)
                    corr = ((double)po.q[g] - rd[K * 32 + lane]) + (df_to_double(acc) - (double)po.m[g]);
            }
            if (!good) {
                atomicOr(err, kErrRange);
            } else {
                const double r = lnL_tmarg[g] + corr;
                if (!isfinite(r))
                    atomicOr(err, kErrNonFinite);
                lnL_tmarg[g] = r;
                if (lnw && lnpw)
                    lnw[g] = r + lnpw[g];
            }
        }
        if (lnL_t) {
            // the per-bin values of the warp's samples move by the same amount
            for (int t = 0; t < nb; ++t) {
                const uint32_t gt = __shfl_sync(0xffffffffu, g, t);
                const double ct = __shfl_sync(0xffffffffu, corr, t);
                if (__shfl_sync(0xffffffffu, good ? 1 : 0, t))
                    for (int j = lane; j < NT; j += 32)
                        lnL_t[(int64_t)gt * NT + j] += ct;
            }
        }
        __syncwarp();
    }
}

cudaError_t launch_fix_prep(const Problem &P, FixTables T, float4 *ua, float4 *vb, float4 *qdf, cudaStream_t st)
{
    const int64_t total = (int64_t)P.K * (T.nA + T.nB) + (int64_t)P.K * P.M * P.n_q;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    fix_prep_kernel<<<grid, 256, 0, st>>>(P.U64, P.V64, P.Q64, P.K, P.M, P.n_q, T, ua, vb, qdf);
    return cudaGetLastError();
}

cudaError_t launch_fix(const Problem &P, BinTable bt, FixTables T, const double *theta, int64_t n, PeakOut po,
                       int blen, float thr, uint32_t *idx, uint32_t *count, double *lnL_tmarg, double *lnL_t,
                       const double *lnpw, double *lnw, int *err, cudaStream_t st, int *launched)
{
    if (n <= 0)
        return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess)
        return e;
    fix_select_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(po.q, po.m, n, thr, idx, count);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one block per SM with as many warps as its shared memory holds (the pair tables are
    // staged once per block, the per-warp scratch grows with the warps): latency-bound
    // double-float chains want the warps
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t wbytes = fix_warp_bytes(P.K, P.M, T.dmax);
    const size_t tbytes = (size_t)P.K * (T.nA + T.nB) * 16 + (size_t)(T.nA + T.nB) * 2;
    int nw = kFixMaxWarps;
    while (nw > 1 && wbytes * nw + tbytes > (size_t)max_smem)
        --nw;
    const int64_t per_block = 32 * nw;
    const int grid = (int)std::min<int64_t>((n + per_block - 1) / per_block, (int64_t)sms);
    const size_t smem = wbytes * nw + tbytes;
    fix_kernel<<<grid, 32 * nw, smem, st>>>(P, bt, T, theta, idx, count, po, blen, lnL_tmarg, lnL_t, lnpw,
                                                    lnw, err);
    if (launched)
        *launched = 2;
    return cudaGetLastError();
}

cudaError_t prepare_fix_kernels() { return allow_max_dynamic_smem(fix_kernel); }

}  // namespace rift
