// Peak-rate microbenchmarks of the units the likelihood kernels use (rift_ile_peak_rate):
// the float32 FMA pipe, the special-function unit's ex2, the float64 FMA pipe, and the
// tcgen05 kind::f16 tensor-core MMA with the A operand in tensor memory (the form the
// tensor-core likelihood kernel issues).  Measured on the
// device with CUDA events, so that roofline fractions are taken against this part's
// measured rates rather than datasheet figures.
#include <algorithm>
#include <cstdint>

#include "../../include/rift_ile.h"
#include "ile_kernels.h"
#include "tc_ptx.cuh"

namespace rift {
namespace {

constexpr int kFmaChains = 8;
constexpr int kFmaThreads = 256;
constexpr int kFmaBlocksPerSm = 4;

// kFmaChains independent FMA chains per thread (latency 4 cycles: 8 chains and 32 warps per
// SM keep the pipe full); the result is written only if it equals an impossible value, so
// the chains stay live.
__global__ void __launch_bounds__(kFmaThreads) peak_fma_kernel(int iters, float *sink)
{
    float a[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c)
        a[c] = 1e-3f * (float)(threadIdx.x + c);
    const float b = 0.9999999f, d = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kFmaChains; ++c)
                a[c] = fmaf(a[c], b, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c)
        s += a[c];
    if (s == -12345.f)
        sink[threadIdx.x] = s;
}

// The same structure for the special-function unit: each chain is x <- 2^(x c), with c < 0
// chosen so that the values stay in a normal range; and for the float64 FMA pipe.
__global__ void __launch_bounds__(kFmaThreads) peak_ex2_kernel(int iters, float *sink)
{
    float a[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c)
        a[c] = 1e-3f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kFmaChains; ++c) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a[c]));
                a[c] = y;
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c)
        s += a[c];
    if (s == -12345.f)
        sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kFmaThreads) peak_dfma_kernel(int iters, double *sink)
{
    double a[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c)
        a[c] = 1e-3 * (double)(threadIdx.x + c);
    const double b = 0.9999999, d = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kFmaChains; ++c)
                a[c] = fma(a[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c)
        s += a[c];
    if (s == -12345.0)
        sink[threadIdx.x] = s;
}

constexpr int kTcPeakThreads = 128;
constexpr uint64_t kPeakWaitNs = 2000000000ull;
// unused dynamic shared memory that admits one CTA per SM (two would exceed the SM's
// 228 KB), so that every SM holds exactly one tensor-memory allocation
constexpr size_t kTcPeakPadSmem = 116 * 1024;

// One CTA per SM.  B: N x 16 float16 (zero) in the canonical K-major no-swizzle layout
// (core matrices of 8 rows x 16 bytes, leading byte offset 128 B, stride byte offset
// 256 B); A: 128 x 16 float16 (zero) in tensor memory at column 256; D: 128 x N float32 at
// column 0.  Thread 0 issues `iters` MMAs back to back (accumulating), commits, and waits
// (bounded) for completion.
__global__ void __launch_bounds__(kTcPeakThreads, 1) peak_tc_kernel(int iters, int n_cols, int *err)
{
    __shared__ __align__(1024) __half Bs[256 * 16];
    __shared__ uint64_t bar;
    __shared__ uint32_t tptr;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < 256 * 16; e += blockDim.x)
        Bs[e] = __float2half_rn(0.f);
    if (warp == 0)
        tc::tmem_alloc(&tptr, 512);
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tptr;
    {
        // A = 0: each warp writes its 32 lanes, 8 columns of two float16 each
        uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        tc::tmem_st8(tmem + ((uint32_t)(32 * warp) << 16) + 256u, z);
        tc::tmem_st_wait();
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0) {
        const uint32_t lo = ((tc::smem_u32(Bs) & 0x3FFFFu) >> 4) | ((128u >> 4) << 16);
        const uint64_t bdesc = ((uint64_t)(((256u >> 4) & 0x3FFFu) | (1u << 14)) << 32) | lo;
        const uint32_t idesc = tc::idesc_f16_f32(128, (uint32_t)n_cols);
        for (int i = 0; i < iters; ++i)
            tc::mma_f16_ta(tmem, tmem + 256u, bdesc, idesc, i > 0 ? 1u : 0u);
        tc::mma_commit(&bar);
        if (!tc::mbar_wait(&bar, 0, kPeakWaitNs)) {
            atomicOr(err, kErrTimeout);
            tc::mbar_wait(&bar, 0, kPeakWaitNs);   // the MMAs in flight, before the columns are freed
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

}  // namespace
}  // namespace rift

using namespace rift;

extern "C" int rift_ile_peak_rate(int32_t what, double *tflops)
{
    if (!tflops || what < RIFT_PEAK_FP32_FMA || what > RIFT_PEAK_FP64_FMA)
        return RIFT_EINVAL;
    const bool tc = what == RIFT_PEAK_TC_F16_N128 || what == RIFT_PEAK_TC_F16_N256;
    int dev = 0, sms = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) {
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    if (tc && major != 10)
        return RIFT_EINVAL;   // tcgen05 needs the sm_100 family
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    int *err = nullptr;
    int rc = RIFT_OK;
    double best = 0.0;
    if ((tc && allow_max_dynamic_smem(peak_tc_kernel) != cudaSuccess) ||
        cudaStreamCreate(&st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMallocAsync(&sink, 8 * kFmaThreads, st) != cudaSuccess ||
        cudaMallocAsync(&err, sizeof(int), st) != cudaSuccess || cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
        rc = RIFT_ECUDA;
    } else {
        // warm-up, then the best of three timed launches
        for (int rep = 0; rep < 4 && rc == RIFT_OK; ++rep) {
            double flop = 0.0;
            cudaEventRecord(e0, st);
            if (what == RIFT_PEAK_FP32_FMA) {
                const int iters = 4096;
                const int blocks = sms * kFmaBlocksPerSm;
                peak_fma_kernel<<<blocks, kFmaThreads, 0, st>>>(iters, sink);
                flop = 2.0 * kFmaChains * 16.0 * iters * (double)blocks * kFmaThreads;
            } else if (what == RIFT_PEAK_EX2) {
                const int iters = 1024;
                const int blocks = sms * kFmaBlocksPerSm;
                peak_ex2_kernel<<<blocks, kFmaThreads, 0, st>>>(iters, sink);
                flop = kFmaChains * 16.0 * iters * (double)blocks * kFmaThreads;   // exponentials
            } else if (what == RIFT_PEAK_FP64_FMA) {
                const int iters = 64;
                const int blocks = sms * kFmaBlocksPerSm;
                peak_dfma_kernel<<<blocks, kFmaThreads, 0, st>>>(iters, reinterpret_cast<double *>(sink));
                flop = 2.0 * kFmaChains * 16.0 * iters * (double)blocks * kFmaThreads;
            } else {
                const int n_cols = what == RIFT_PEAK_TC_F16_N128 ? 128 : 256;
                const int iters = 16384;
                peak_tc_kernel<<<sms, kTcPeakThreads, kTcPeakPadSmem, st>>>(iters, n_cols, err);
                flop = 2.0 * 128.0 * n_cols * 16.0 * iters * (double)sms;
            }
            cudaEventRecord(e1, st);
            int herr = 0;
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = RIFT_ECUDA;
            } else if (herr) {
                rc = RIFT_ETIMEOUT;
            } else if (rep > 0 && ms > 0.f) {
                best = std::max(best, flop / (ms * 1e-3) / 1e12);
            }
        }
    }
    if (sink)
        cudaFreeAsync(sink, st);
    if (err)
        cudaFreeAsync(err, st);
    if (st)
        cudaStreamSynchronize(st);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (st)
        cudaStreamDestroy(st);
    cudaGetLastError();
    *tflops = best;
    return rc;
}
