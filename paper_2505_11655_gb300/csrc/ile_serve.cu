// Serving loop for many ILE solves (include/rift_ile.h, rift_srv_*): arrival-order
// admission by device footprint and free slot, one host worker and CUDA stream per
// slot, so that solves admitted while others run overlap on the GPU.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rift_ile.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    rift_ile_config cfg{};
    std::vector<double> det_tensor, det_pos, q_t0, Q, U, V;
    std::vector<int32_t> lm;
    int32_t n_iter = 1;
    int64_t n_per_iter = 0;
    uint64_t tag = 0;
    int64_t footprint = 0;
    double t_submit = 0;
};

}  // namespace

struct rift_srv {
    rift_srv_config cfg{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Request>> queue;
    std::deque<rift_srv_completion> done;
    int64_t active_bytes = 0;
    int32_t active = 0;
    bool stop = false;
    int device = 0;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

int run_one(cudaStream_t st, Request &r, rift_ile_result *res)
{
    rift_ile_t *h = nullptr;
    int rc = rift_ile_create(&r.cfg, st, &h);
    if (rc == RIFT_OK)
        rc = rift_ile_set_overlaps(h, r.Q.data(), r.U.data(), r.V.data(), RIFT_MEM_HOST);
    if (rc == RIFT_OK)
        rc = rift_ile_adapt(h, r.n_iter, r.n_per_iter, res);
    rift_ile_destroy(h);
    return rc;
}

void worker(rift_srv *s, int slot)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::unique_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop ||
                       (!s->queue.empty() && s->active_bytes + s->queue.front()->footprint <= s->cfg.hbm_budget_bytes);
            });
            if (s->stop)
                return;
            r = std::move(s->queue.front());
            s->queue.pop_front();
            s->active_bytes += r->footprint;
            s->active += 1;
        }
        rift_srv_completion c{};
        c.tag = r->tag;
        c.t_submit_ms = r->t_submit;
        c.t_admit_ms = s->now_ms();
        c.status = run_one(s->streams[slot], *r, &c.result);
        c.t_done_ms = s->now_ms();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->active_bytes -= r->footprint;
            s->active -= 1;
            s->done.push_back(c);
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

int rift_srv_create(const rift_srv_config *cfg, rift_srv_t **out)
{
    if (!out)
        return RIFT_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->hbm_budget_bytes <= 0)
        return RIFT_EINVAL;
    auto s = std::make_unique<rift_srv>();
    s->cfg = *cfg;
    s->t0 = Clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    for (int i = 0; i < cfg->max_slots; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : s->streams)
                cudaStreamDestroy(x);
            return RIFT_ECUDA;
        }
        s->streams.push_back(st);
    }
    for (int i = 0; i < cfg->max_slots; ++i)
        s->workers.emplace_back(worker, s.get(), i);
    *out = s.release();
    return RIFT_OK;
}

int rift_srv_submit(rift_srv_t *s, const rift_srv_request *req)
{
    if (!s || !req || !req->cfg || !req->Q || !req->U || !req->V || req->n_iter < 1 || req->n_iter > RIFT_MAX_ITER ||
        req->n_per_iter < 1 || req->n_per_iter > req->cfg->max_samples)
        return RIFT_EINVAL;
    const int64_t fp = rift_ile_footprint(req->cfg);
    if (fp < 0)
        return RIFT_EINVAL;
    if (fp > s->cfg.hbm_budget_bytes)
        return RIFT_ENOMEM;
    auto r = std::make_unique<Request>();
    const rift_ile_config &c = *req->cfg;
    const size_t K = c.n_det, M = c.n_modes;
    r->cfg = c;
    r->det_tensor.assign(c.det_tensor, c.det_tensor + 9 * K);
    r->det_pos.assign(c.det_pos_m, c.det_pos_m + 3 * K);
    r->q_t0.assign(c.q_t0_s, c.q_t0_s + K);
    r->lm.assign(c.lm, c.lm + 2 * M);
    const double *Q = static_cast<const double *>(req->Q), *U = static_cast<const double *>(req->U),
                 *V = static_cast<const double *>(req->V);
    r->Q.assign(Q, Q + 2 * K * M * (size_t)c.n_q);
    r->U.assign(U, U + 2 * K * M * M);
    r->V.assign(V, V + 2 * K * M * M);
    r->cfg.det_tensor = r->det_tensor.data();
    r->cfg.det_pos_m = r->det_pos.data();
    r->cfg.q_t0_s = r->q_t0.data();
    r->cfg.lm = r->lm.data();
    r->n_iter = req->n_iter;
    r->n_per_iter = req->n_per_iter;
    r->tag = req->tag;
    r->footprint = fp;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->t_submit = s->now_ms();
        s->queue.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return RIFT_OK;
}

int rift_srv_poll(rift_srv_t *s, rift_srv_completion *out, int32_t max, int32_t timeout_ms, int32_t *n_out)
{
    if (!s || !out || max < 1 || !n_out)
        return RIFT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done.empty(); });
    int32_t n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    return RIFT_OK;
}

int rift_srv_pending(rift_srv_t *s, int32_t *queued, int32_t *active)
{
    if (!s)
        return RIFT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued)
        *queued = (int32_t)s->queue.size();
    if (active)
        *active = s->active;
    return RIFT_OK;
}

void rift_srv_destroy(rift_srv_t *s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers)
        t.join();
    for (cudaStream_t st : s->streams)
        cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
