// Batch executor (include/rift_ile.h, rift_batch_*): many independent solves as one
// CUDA graph.
//
// Each solve's whole adaptive sequence is captured on the batch's private capture
// stream into a graph of its own (the same enqueue path rift_ile_adapt uses, without
// stage timers) and added to the batch graph as a child node with no dependencies, so
// the solves are parallel branches.  A gather kernel, dependent on every branch,
// packs each solve's error word, pooled record and per-iteration records into one
// buffer that a single copy brings back.  Later runs replay the instantiated graph:
// the sampler iteration counters advance on the device, so every run continues each
// solve's adaptive sequence.
#include <cstring>
#include <new>
#include <set>
#include <vector>

#include "ile_handle.h"

using namespace rift;
using namespace rift::host;

namespace {

struct BatchSrc {
    const int *err;
    const double *final_out;   // [6]
    const double *stats;       // [8 * n_iter]
    int n_iter;
};

// out[i] = { err word, final[0..6), stats[0 .. 8 n_iter) } with row stride `stride`
__global__ void gather_kernel(const BatchSrc *__restrict__ src, int n, double *__restrict__ out, int stride)
{
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const BatchSrc s = src[i];
        double *o = out + (size_t)i * stride;
        const int rec = 7 + 8 * s.n_iter;
        for (int e = threadIdx.x; e < rec; e += blockDim.x) {
            double v;
            if (e == 0)
                v = (double)*s.err;
            else if (e < 7)
                v = s.final_out[e - 1];
            else
                v = s.stats[e - 7];
            o[e] = v;
        }
    }
}

}  // namespace

struct rift_batch {
    std::vector<rift_ile_t *> h;
    std::vector<int32_t> n_iter;
    std::vector<int64_t> n;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<LaunchPlan> plans;   // plans the graph was captured with
    std::vector<int64_t> solve_launches;   // kernels of each solve's branch
    BatchSrc *src_dev = nullptr;
    double *out_dev = nullptr, *out_host = nullptr;
    int stride = 0;
    int64_t launches = -1;
};

namespace {

void batch_release(rift_batch *b)
{
    if (!b)
        return;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->src_dev)
        cudaFree(b->src_dev);
    if (b->out_dev)
        cudaFree(b->out_dev);
    if (b->out_host)
        cudaFreeHost(b->out_host);
    if (b->t0)
        cudaEventDestroy(b->t0);
    if (b->t1)
        cudaEventDestroy(b->t1);
    if (b->cap_stream)
        cudaStreamDestroy(b->cap_stream);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

// Capture solve i's adaptive sequence as a graph of its own.
int capture_solve(rift_batch *b, int i, cudaGraph_t *out, int64_t *launches)
{
    rift_ile_t *h = b->h[i];
    cudaStream_t saved = h->stream;
    const bool saved_timed = h->timed;
    h->stream = b->cap_stream;
    h->timed = false;
    const int64_t l0 = h->launches;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = RIFT_ECUDA;
    if (e == cudaSuccess) {
        h->capturing = true;
        rc = enqueue_adapt(h, b->n_iter[i], b->n[i]);
        h->capturing = false;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc == RIFT_OK && e != cudaSuccess)
            rc = RIFT_ECUDA;
        if (rc == RIFT_OK)
            *out = g;
        else if (g)
            cudaGraphDestroy(g);
    }
    *launches = h->launches - l0;
    h->launches = l0;
    h->stream = saved;
    h->timed = saved_timed;
    cudaGetLastError();
    return rc;
}

int build_graph(rift_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const int n = (int)b->h.size();
    cudaGraph_t parent = nullptr;
    CK(cudaGraphCreate(&parent, 0));
    std::vector<cudaGraphNode_t> branches(n);
    std::vector<int64_t> per_solve(n, 0);
    int64_t launches = 0;
    int rc = RIFT_OK;
    for (int i = 0; i < n && rc == RIFT_OK; ++i) {
        cudaGraph_t g = nullptr;
        int64_t l = 0;
        rc = capture_solve(b, i, &g, &l);
        if (rc != RIFT_OK)
            break;
        launches += l;
        per_solve[i] = l;
        if (cudaGraphAddChildGraphNode(&branches[i], parent, nullptr, 0, g) != cudaSuccess)
            rc = RIFT_ECUDA;
        cudaGraphDestroy(g);
    }
    if (rc == RIFT_OK) {
        // the gather, after every branch
        cudaKernelNodeParams kp{};
        const BatchSrc *src = b->src_dev;
        int cnt = n;
        double *out = b->out_dev;
        int stride = b->stride;
        void *args[] = {&src, &cnt, &out, &stride};
        kp.func = (void *)gather_kernel;
        kp.gridDim = dim3(n < 1024 ? n : 1024);
        kp.blockDim = dim3(128);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t gather;
        if (cudaGraphAddKernelNode(&gather, parent, branches.data(), (size_t)n, &kp) != cudaSuccess)
            rc = RIFT_ECUDA;
        launches += 1;
    }
    if (rc == RIFT_OK && cudaGraphInstantiate(&b->exec, parent, 0) != cudaSuccess) {
        b->exec = nullptr;
        rc = RIFT_ECUDA;
    }
    cudaGraphDestroy(parent);
    cudaGetLastError();
    if (rc == RIFT_OK) {
        b->launches = launches;
        b->solve_launches = per_solve;
        b->plans.resize(n);
        for (int i = 0; i < n; ++i)
            b->plans[i] = b->h[i]->plan;
    }
    return rc;
}

}  // namespace

extern "C" {

int rift_batch_create(rift_ile_t *const *solves, int32_t n, const int32_t *n_iter, const int64_t *n_per_iter,
                      void *cuda_stream, rift_batch_t **out)
{
    if (!out)
        return RIFT_EINVAL;
    *out = nullptr;
    if (!solves || !n_iter || !n_per_iter || n < 1 || n > 65536)
        return RIFT_EINVAL;
    std::set<const rift_ile_t *> seen;
    int32_t max_iter = 0;
    for (int i = 0; i < n; ++i) {
        const rift_ile_t *h = solves[i];
        if (!h || !seen.insert(h).second || n_iter[i] < 1 || n_iter[i] > RIFT_MAX_ITER || n_per_iter[i] < 1 ||
            n_per_iter[i] > h->cap)
            return RIFT_EINVAL;
        max_iter = n_iter[i] > max_iter ? n_iter[i] : max_iter;
    }
    for (int i = 0; i < n; ++i)
        if (!solves[i]->have_overlaps)
            return RIFT_ESTATE;
    rift_batch *b = new (std::nothrow) rift_batch();
    if (!b)
        return RIFT_ENOMEM;
    b->h.assign(solves, solves + n);
    b->n_iter.assign(n_iter, n_iter + n);
    b->n.assign(n_per_iter, n_per_iter + n);
    b->stride = 7 + 8 * max_iter;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!b->stream) {
        if (cudaStreamCreate(&b->stream) != cudaSuccess) {
            b->stream = nullptr;
            batch_release(b);
            return RIFT_ECUDA;
        }
        b->own_stream = true;
    }
    std::vector<BatchSrc> src(n);
    for (int i = 0; i < n; ++i)
        src[i] = BatchSrc{solves[i]->err, solves[i]->final_out, solves[i]->stats, n_iter[i]};
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess ||
        cudaMalloc(&b->src_dev, sizeof(BatchSrc) * n) != cudaSuccess ||
        cudaMalloc(&b->out_dev, sizeof(double) * (size_t)n * b->stride) != cudaSuccess ||
        cudaMallocHost(&b->out_host, sizeof(double) * (size_t)n * b->stride) != cudaSuccess ||
        cudaMemcpyAsync(b->src_dev, src.data(), sizeof(BatchSrc) * n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        batch_release(b);
        return RIFT_ECUDA;
    }
    *out = b;
    return RIFT_OK;
}

int rift_batch_run(rift_batch_t *b, rift_ile_result *out)
{
    if (!b || !out)
        return RIFT_EINVAL;
    const int n = (int)b->h.size();
    // plans first (timed candidates for classes not seen yet), outside any capture;
    // the batch is ordered after whatever each handle's stream still holds
    bool rebuild = !b->exec;
    for (int i = 0; i < n; ++i) {
        rift_ile_t *h = b->h[i];
        if (!h->have_overlaps)
            return RIFT_ESTATE;
        RK(choose_plan(h, b->n[i]));
        CK(cudaStreamSynchronize(h->stream));
        if (!rebuild && b->plans[i] != h->plan)
            rebuild = true;
    }
    if (rebuild)
        RK(build_graph(b));
    CK(cudaEventRecord(b->t0, b->stream));
    CK(cudaGraphLaunch(b->exec, b->stream));
    CK(cudaEventRecord(b->t1, b->stream));
    CK(cudaMemcpyAsync(b->out_host, b->out_dev, sizeof(double) * (size_t)n * b->stride, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, b->t0, b->t1);
    int first = RIFT_OK;
    for (int i = 0; i < n; ++i) {
        rift_ile_t *h = b->h[i];
        const double *o = b->out_host + (size_t)i * b->stride;
        const int rc = map_err((int)o[0]);
        rift_ile_result &r = out[i];
        std::memset(&r, 0, sizeof(r));
        r.lnZ = o[1];
        r.sigma_lnZ = o[2];
        r.n_eff = o[3];
        r.n_ess = o[4];
        r.lnL_max = o[5];
        r.n_total = (int64_t)o[6];
        r.n_iter = b->n_iter[i];
        r.status = rc;
        for (int g = 0; g < b->n_iter[i]; ++g) {
            const double *s = o + 7 + 8 * g;
            r.lnZ_iter[g] = s[0];
            r.sigma_iter[g] = s[1];
            r.n_eff_iter[g] = s[2];
            r.n_ess_iter[g] = s[3];
        }
        r.time_ms[3] = ms;
        h->iteration += (uint32_t)b->n_iter[i];
        h->last_n = b->n[i];
        h->launches += b->solve_launches[i];
        if (first == RIFT_OK && rc != RIFT_OK)
            first = rc;
    }
    return first;
}

int64_t rift_batch_kernel_launches(const rift_batch_t *b) { return b ? b->launches : -1; }

void rift_batch_destroy(rift_batch_t *b) { batch_release(b); }

}  // extern "C"
