// Launch autotuner of the float32 likelihood stage.
//
// Which tile kernel wins (128-sample tensor-core tiles or 64-sample CUDA-core tiles)
// and how densely the sky sort fills its Hilbert cells depend on the problem class:
// the detector count, the mode count (padded to the 16-wide MMA K step), the time
// grid, the Q length, the batch size and whether the distance is marginalised, and on how
// far the sampler has adapted (the samples of an adapted sampler crowd into fewer sky
// cells and delays, which changes the best sort).  The first batch of a class times every candidate plan on samples drawn
// from the sampler (keys + sort + likelihood, best of two runs) and the winner is cached
// for the process.  A handle whose sampler has adapted twice or more, on a batch of 2^19
// samples or more, looks up a second class whose tensor-core plans (sky-cell fill, sort
// key) are timed the same way on its first adapted batch (a class whose first plan is the
// CUDA-core kernel keeps it).  The plan thus depends only on the problem class and on
// whether the handle has adapted twice, never on another handle's history.  With
// RIFT_ILE_TUNE_CACHE set to a file path the cache is also read from and appended to that
// file.
#include <cmath>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "ile_handle.h"

namespace rift {
namespace host {
namespace {

constexpr int64_t kTuneMinBatch = 4096;   // smaller batches take the untuned default
constexpr uint32_t kAdaptedAfter = 2;      // iterations after which a sampler counts as adapted
constexpr int64_t kAdaptedMinBatch = 1 << 19;   // smaller batches keep their first plan

struct TuneCache {
    std::mutex mu;
    std::map<std::string, LaunchPlan> plans;
    bool loaded = false;
};

TuneCache &cache()
{
    static TuneCache c;
    return c;
}

const char *cache_path()
{
    const char *p = std::getenv("RIFT_ILE_TUNE_CACHE");
    return p && p[0] ? p : nullptr;
}

// caller holds the lock
void load_file(TuneCache &c)
{
    if (c.loaded)
        return;
    c.loaded = true;
    const char *path = cache_path();
    if (!path)
        return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string key;
        LaunchPlan p;
        if ((is >> key >> p.tc >> p.per_cell) && (p.tc == 0 || p.tc == 1) && p.per_cell >= 1 && p.per_cell <= 64) {
            if (!(is >> p.delay3) || (p.delay3 != 0 && p.delay3 != 1))
                p.delay3 = 0;
            c.plans[key] = p;
        }
    }
}

void append_file(const std::string &key, const LaunchPlan &p)
{
    const char *path = cache_path();
    if (!path)
        return;
    std::ofstream f(path, std::ios::app);
    f << key << ' ' << p.tc << ' ' << p.per_cell << ' ' << p.delay3 << '\n';
}

std::string class_key(const rift_ile_t *h, int64_t n)
{
    const int kp = (2 * h->prob.M + 15) / 16;
    const int nb = (int)std::floor(std::log2((double)n) / 2.0);   // batch size in factors of 4
    std::ostringstream s;
    s << "K" << h->prob.K << "_kp" << kp << "_nt" << h->prob.n_t << "_nq" << h->prob.n_q << "_n4^" << nb;
    if (h->prob.dist_marg)   // the distance-marginalised instance is a kernel of its own
        s << "_dm";
    return s.str();
}

// Time keys + sort + likelihood for one plan on the drawn batch (best of two).
int time_plan(rift_ile_t *h, int64_t n, const LaunchPlan &p, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    h->plan = p;
    RK(grid_for_batch(h, n));
    float best = INFINITY;
    for (int rep = 0; rep < 2; ++rep) {
        CK(cudaEventRecord(e0, h->stream));
        CK(launch_keys(h->grid, h->theta, n, h->key, h->stream));
        CK(launch_sort(h->grid, h->key, n, h->sort_scratch, h->perm, h->stream));
        CK(launch_tiled(h, h->theta, n, h->lnL, nullptr, nullptr, nullptr));
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0;
        CK(cudaEventElapsedTime(&t, e0, e1));
        best = t < best ? t : best;
    }
    *ms = best;
    return RIFT_OK;
}

int measure(rift_ile_t *h, int64_t n, LaunchPlan *out, bool tc_only)
{
    // CUDA-core tiles; tensor-core tiles at three sky-cell fills; with three or more
    // detectors also tensor-core tiles sorted by a Morton key of three delays (fewer
    // tile sub-groups at low sample density).  tc_only: the tensor-core plans alone.
    static const LaunchPlan candidates[] = {{0, 4, 0}, {1, 2, 0}, {1, 4, 0}, {1, 8, 0}, {1, 4, 1}};
    const int n_cand = h->prob.K >= 3 ? 5 : 4;
    h->plan = LaunchPlan{};
    RK(grid_for_batch(h, n));
    CK(launch_draw(sampler_of(h), h->grid, h->iter_dev, 0, n, h->theta, h->lnpw, h->bins, h->key, h->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaGetLastError();
        return RIFT_ECUDA;
    }
    float best = INFINITY;
    int rc = RIFT_OK;
    for (int ci = tc_only ? 1 : 0; ci < n_cand; ++ci) {
        const LaunchPlan &p = candidates[ci];
        float t = 0;
        rc = time_plan(h, n, p, e0, e1, &t);
        if (rc != RIFT_OK)
            break;
        if (t < best) {
            best = t;
            *out = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timing runs may have flagged samples of the scratch batch; the real
    // iteration redraws the same batch and resets the flags
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return rc;
}

}  // namespace

namespace {

// RIFT_ILE_DELAY3=0/1 forces the sort key of three-detector problems.
void apply_sort_override(rift_ile_t *h)
{
    const char *env = std::getenv("RIFT_ILE_DELAY3");
    if (env && (env[0] == '0' || env[0] == '1'))
        h->plan.delay3 = (env[0] == '1' && h->prob.K >= 3) ? 1 : 0;
}

int choose_plan_tuned(rift_ile_t *h, int64_t n, bool measure_allowed);

}  // namespace

int choose_plan(rift_ile_t *h, int64_t n, bool measure_allowed)
{
    const int rc = choose_plan_tuned(h, n, measure_allowed);
    apply_sort_override(h);
    return rc;
}

namespace {

int choose_plan_tuned(rift_ile_t *h, int64_t n, bool measure_allowed)
{
    if (!use_fp32(h))
        return RIFT_OK;
    if (!h->tc_ok || h->tc_mode == 0) {
        h->plan = LaunchPlan{0, 4, 0};
        return RIFT_OK;
    }
    if (h->tc_mode == 1) {
        h->plan = LaunchPlan{1, 4, 0};
        return RIFT_OK;
    }
    // an adapted sampler's large batch re-tunes the tensor-core plan (sky-cell fill and sort
    // key) once per class; the kernel family stays that of the first plan
    const std::string base = class_key(h, n);
    const bool adapted = h->iteration >= kAdaptedAfter && n >= kAdaptedMinBatch;
    const std::string key = adapted ? base + "_adapted" : base;
    TuneCache &c = cache();
    bool tc_only = false;
    {
        std::lock_guard<std::mutex> lock(c.mu);
        load_file(c);
        auto it = c.plans.find(key);
        if (it != c.plans.end()) {
            h->plan = it->second;
            return RIFT_OK;
        }
        if (adapted) {
            auto first = c.plans.find(base);
            if (first != c.plans.end()) {
                if (first->second.tc != 1) {   // CUDA-core tiles: nothing to re-tune
                    h->plan = first->second;
                    return RIFT_OK;
                }
                tc_only = true;
            }
        }
    }
    const char *env = std::getenv("RIFT_ILE_TUNE");
    if (!measure_allowed || n < kTuneMinBatch || (env && env[0] == '0')) {
        h->plan = LaunchPlan{};   // untuned default (kernel by batch size)
        return RIFT_OK;
    }
    LaunchPlan best{};
    RK(measure(h, n, &best, tc_only));
    {
        std::lock_guard<std::mutex> lock(c.mu);
        if (c.plans.emplace(key, best).second)
            append_file(key, best);
        h->plan = c.plans[key];
    }
    return RIFT_OK;
}

}  // namespace

}  // namespace host
}  // namespace rift
