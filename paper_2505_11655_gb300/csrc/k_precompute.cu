// Overlaps Q, U, V from frequency-domain inputs (arXiv:2505.11655, Sec. II A, Eq. QUV):
// on a mirror-symmetric two-sided grid f_j with inverse-PSD weights w_k(f), shared mode
// waveforms h_lm(f) and per-detector data d_k(f),
//   Q_k,lm(t_s)   = 2 sum_j w_k(f_j) exp(2 pi i f_j t_s) conj(h_lm(f_j)) d_k(f_j),
//                   t_s = q_t0_k + s / f_s on each detector's Q grid;
//   U_k,lm,l'm'   = 2 sum_j w_k conj(h_lm) h_l'm',   V_k,lm,l'm' = 2 sum_j w_k h_lm(-f_j) h_l'm'(f_j).
// U is Hermitian and V symmetric (the weights are symmetric in f), so only pairs
// lm <= l'm' are summed and mirrored (the halving the paper describes for U and V).
// All in float64.
//
// Q by a fast Fourier transform.  When the frequencies lie on a lattice f_j = f_0 + n_j df
// (integers n_j spanning fewer than L = f_s / df points, L a power of two), then with
// t_s = q_t0 + s / f_s,
//   exp(2 pi i f_j t_s) = exp(2 pi i f_j q_t0) exp(2 pi i f_0 s / f_s) exp(2 pi i n_j s / L),
// so Q_k,lm(t_s) = exp(2 pi i f_0 s / f_s) Y[s mod L], Y the length-L transform (sign +)
// of X[n_j] = A_j exp(2 pi i f_j q_t0): O(L log L) per (detector, mode) instead of
// O(n_q F).  The transform is a radix-2 Stockham (self-sorting) FFT, one kernel per
// stage over every (detector, mode) sequence at once, twiddles exp(2 pi i e / L) from a
// table.  Grids off a lattice (or with L not a power of two) take the direct sum.
#include <algorithm>
#include <cmath>

#include "ile_kernels.h"

namespace rift {

constexpr int kPcThreads = 128;   // Q samples per block
constexpr int kPcChunk = 64;      // frequencies staged per pass

// A[k][m][j] = 2 w_k(f_j) conj(h_m(f_j)) d_k(f_j)
__global__ void qfreq_kernel(const double2 *__restrict__ h, const double2 *__restrict__ d,
                             const double *__restrict__ w, int K, int M, int F, double2 *__restrict__ A)
{
    const int64_t total = (int64_t)K * M * F;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % F), m = (int)((e / F) % M), k = (int)(e / ((int64_t)F * M));
        const double2 hm = h[(size_t)m * F + j], dk = d[(size_t)k * F + j];
        const double s = 2.0 * w[(size_t)k * F + j];
        // conj(h) d
        A[e] = make_double2(s * (hm.x * dk.x + hm.y * dk.y), s * (hm.x * dk.y - hm.y * dk.x));
    }
}

// One thread per (detector, Q sample); all modes accumulated together.
__global__ void __launch_bounds__(kPcThreads) q_series_kernel(const double2 *__restrict__ A,
                                                              const double *__restrict__ f, int K, int M, int F,
                                                              const double *__restrict__ q_t0, double fs, int n_q,
                                                              double2 *__restrict__ Q)
{
    __shared__ double2 sA[kMaxModes * kPcChunk];
    __shared__ double sf[kPcChunk];
    const int k = blockIdx.y;
    const int s = blockIdx.x * kPcThreads + threadIdx.x;
    const double t = q_t0[k] + (double)s / fs;
    double re[kMaxModes], im[kMaxModes];
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m)
        re[m] = im[m] = 0.0;
    for (int j0 = 0; j0 < F; j0 += kPcChunk) {
        const int nj = min(kPcChunk, F - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < M * kPcChunk; e += kPcThreads) {
            const int m = e / kPcChunk, j = e % kPcChunk;
            sA[e] = j < nj ? A[((size_t)k * M + m) * F + j0 + j] : make_double2(0.0, 0.0);
        }
        for (int j = threadIdx.x; j < kPcChunk; j += kPcThreads)
            sf[j] = j < nj ? f[j0 + j] : 0.0;
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
            double sn, cs;
            sincospi(2.0 * sf[j] * t, &sn, &cs);
#pragma unroll
            for (int m = 0; m < kMaxModes; ++m) {
                if (m < M) {
                    const double2 a = sA[m * kPcChunk + j];
                    re[m] += a.x * cs - a.y * sn;
                    im[m] += a.x * sn + a.y * cs;
                }
            }
        }
    }
    if (s < n_q) {
#pragma unroll
        for (int m = 0; m < kMaxModes; ++m)
            if (m < M)
                Q[((size_t)k * M + m) * n_q + s] = make_double2(re[m], im[m]);
    }
}

// One warp per (detector, pair a <= b): U and V, mirrored.
__global__ void uv_kernel(const double2 *__restrict__ h, const double *__restrict__ w, int K, int M, int F,
                          double2 *__restrict__ U, double2 *__restrict__ V)
{
    const int lane = threadIdx.x & 31;
    const int pairs = M * (M + 1) / 2;
    const int64_t total = (int64_t)K * pairs;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < total; e += warps) {
        const int k = (int)(e / pairs);
        int p = (int)(e % pairs), a = 0;
        while (p >= M - a) {   // pair index -> (a, b), a <= b
            p -= M - a;
            ++a;
        }
        const int b = a + p;
        double ur = 0, ui = 0, vr = 0, vi = 0;
        for (int j = lane; j < F; j += 32) {
            const double wj = 2.0 * w[(size_t)k * F + j];
            const double2 ha = h[(size_t)a * F + j], hb = h[(size_t)b * F + j];
            const double2 hm = h[(size_t)a * F + (F - 1 - j)];   // h_a(-f_j)
            ur += wj * (ha.x * hb.x + ha.y * hb.y);
            ui += wj * (ha.x * hb.y - ha.y * hb.x);
            vr += wj * (hm.x * hb.x - hm.y * hb.y);
            vi += wj * (hm.x * hb.y + hm.y * hb.x);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ur += __shfl_xor_sync(0xffffffffu, ur, o);
            ui += __shfl_xor_sync(0xffffffffu, ui, o);
            vr += __shfl_xor_sync(0xffffffffu, vr, o);
            vi += __shfl_xor_sync(0xffffffffu, vi, o);
        }
        if (a == b)
            ui = 0.0;   // w |h|^2 is real (the fused products leave a rounding residual)
        if (lane == 0) {
            const size_t ab = ((size_t)k * M + a) * M + b, ba = ((size_t)k * M + b) * M + a;
            U[ab] = make_double2(ur, ui);
            U[ba] = make_double2(ur, -ui);
            V[ab] = make_double2(vr, vi);
            V[ba] = make_double2(vr, vi);
        }
    }
}

// ---------------------------------------------------------------- FFT path for Q

// T[e] = exp(2 pi i e / L), e < L / 2
__global__ void fft_twiddle_kernel(int L, double2 *__restrict__ T)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L / 2; e += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)e / (double)L, &sn, &cs);
        T[e] = make_double2(cs, sn);
    }
}

// X [K M][L] (zeroed): X[km][n_j] = A[km][j] exp(2 pi i f_j q_t0_k)
__global__ void fft_scatter_kernel(const double2 *__restrict__ A, const double *__restrict__ f,
                                   const int *__restrict__ nidx, int K, int M, int F, const double *__restrict__ q_t0,
                                   int L, double2 *__restrict__ X)
{
    const int64_t total = (int64_t)K * M * F;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % F);
        const int64_t km = e / F;
        const int k = (int)(km / M);
        double sn, cs;
        sincospi(2.0 * f[j] * q_t0[k], &sn, &cs);
        const double2 a = A[e];
        X[km * L + nidx[j]] = make_double2(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
    }
}

// One radix-2 Stockham stage (sub-transforms of length Ns combined into 2 Ns) of every
// sequence: butterfly j < L/2 of a sequence reads j and j + L/2 and writes
// (j / Ns) 2 Ns + j % Ns and that plus Ns, with twiddle exp(2 pi i (j % Ns) / (2 Ns)).
__global__ void fft_stage_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int L, int Ns,
                                 const double2 *__restrict__ T, int64_t n_seq)
{
    const int half = L >> 1;
    const int64_t total = n_seq * half;
    const int tstride = half / Ns;   // T index step: (j % Ns) L / (2 Ns)
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / half;
        const int j = (int)(e - q * half);
        const int kk = j & (Ns - 1);
        const double2 w = T[(size_t)kk * tstride];
        const double2 a = in[q * L + j], b0 = in[q * L + j + half];
        const double2 b = make_double2(b0.x * w.x - b0.y * w.y, b0.x * w.y + b0.y * w.x);
        const int64_t o = q * L + (int64_t)(j / Ns) * 2 * Ns + kk;
        out[o] = make_double2(a.x + b.x, a.y + b.y);
        out[o + Ns] = make_double2(a.x - b.x, a.y - b.y);
    }
}

// Q[km][s] = exp(2 pi i f_0 s / f_s) Y[km][s mod L]
__global__ void fft_extract_kernel(const double2 *__restrict__ Y, int64_t n_seq, int L, double f0, double fs, int n_q,
                                   double2 *__restrict__ Q)
{
    const int64_t total = n_seq * n_q;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t km = e / n_q;
        const int s = (int)(e - km * n_q);
        double sn, cs;
        sincospi(2.0 * f0 * ((double)s / fs), &sn, &cs);
        const double2 y = Y[km * L + (s & (L - 1))];
        Q[e] = make_double2(y.x * cs - y.y * sn, y.x * sn + y.y * cs);
    }
}

cudaError_t launch_precompute(const double2 *h, const double2 *d, const double *w, const double *f, int K, int M,
                              int F, const double *q_t0_dev, double fs, int n_q, double2 *A_scratch, double2 *Q,
                              double2 *U, double2 *V, cudaStream_t st, const FftPlan *fft, int *launched)
{
    const int64_t nA = (int64_t)K * M * F;
    int k = 0;
    qfreq_kernel<<<(int)std::min<int64_t>((nA + 255) / 256, 152 * 8), 256, 0, st>>>(h, d, w, K, M, F, A_scratch);
    ++k;
    if (fft) {
        const int L = fft->L;
        const int64_t nseq = (int64_t)K * M;
        cudaError_t e = cudaMemsetAsync(fft->X, 0, sizeof(double2) * (size_t)nseq * L, st);
        if (e != cudaSuccess)
            return e;
        fft_twiddle_kernel<<<std::max(1, std::min(L / 2 / 256, 152 * 8)), 256, 0, st>>>(L, fft->T);
        fft_scatter_kernel<<<(int)std::min<int64_t>((nA + 255) / 256, 152 * 8), 256, 0, st>>>(
            A_scratch, f, fft->nidx, K, M, F, q_t0_dev, L, fft->X);
        double2 *a = fft->X, *b = fft->Y;
        const int64_t nb = nseq * (L / 2);
        for (int Ns = 1; Ns < L; Ns <<= 1) {
            fft_stage_kernel<<<(int)std::min<int64_t>((nb + 255) / 256, 152 * 16), 256, 0, st>>>(a, b, L, Ns, fft->T,
                                                                                                 nseq);
            std::swap(a, b);
            ++k;
        }
        const int64_t nqt = nseq * n_q;
        fft_extract_kernel<<<(int)std::min<int64_t>((nqt + 255) / 256, 152 * 8), 256, 0, st>>>(a, nseq, L, fft->f0,
                                                                                              fs, n_q, Q);
        k += 3;
    } else {
        dim3 grid((n_q + kPcThreads - 1) / kPcThreads, K);
        q_series_kernel<<<grid, kPcThreads, 0, st>>>(A_scratch, f, K, M, F, q_t0_dev, fs, n_q, Q);
        ++k;
    }
    const int64_t pairs = (int64_t)K * M * (M + 1) / 2;
    uv_kernel<<<(int)std::min<int64_t>((pairs + 7) / 8, 152 * 8), 256, 0, st>>>(h, w, K, M, F, U, V);
    if (launched)
        *launched = k + 1;
    return cudaGetLastError();
}

}  // namespace rift
