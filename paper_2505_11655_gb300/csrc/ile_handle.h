// The ILE handle and the host-side steps shared by the single-solve entry points
// (ile_api.cu), the batch executor (ile_batch.cu) and the launch autotuner
// (ile_tune.cu).  Internal: nothing here crosses the C ABI.
#pragma once

#include <array>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ile_kernels.h"

// Launch plan of the float32 likelihood stage: which kernel, and how densely the
// sky-sort grid is filled.  Chosen by the autotuner per problem class, or forced by
// RIFT_ILE_TC.
struct LaunchPlan {
    int tc = -1;         // 1 tensor-core tiles, 0 CUDA-core tiles, -1 not chosen yet
    int per_cell = 4;    // samples per Hilbert sky cell
    int delay3 = 0;      // three or more detectors: 1 sorts by a Morton key of three delays
    bool operator==(const LaunchPlan &o) const { return tc == o.tc && per_cell == o.per_cell && delay3 == o.delay3; }
    bool operator!=(const LaunchPlan &o) const { return !(*this == o); }
};

struct rift_ile {
    rift_ile_config cfg{};
    std::vector<double> det_tensor, det_pos, q_t0;
    std::vector<int32_t> lm;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    rift::Problem prob{};
    bool have_overlaps = false;
    int64_t cap = 0;           // samples per device batch
    // overlaps
    double2 *Q64 = nullptr, *U64 = nullptr, *V64 = nullptr;
    float *Qr32 = nullptr;
    float2 *U32 = nullptr, *V32 = nullptr;
    __half *Ttc = nullptr;   // template matrices for the tensor-core kernel (see Problem::Ttc)
    int *tt_exp = nullptr;
    int *bin_i = nullptr;
    float *bin_f = nullptr;
    // per-sample buffers
    double *theta = nullptr, *lnpw = nullptr, *lnL = nullptr, *lnw = nullptr;
    uint64_t *bins = nullptr;
    uint32_t *key = nullptr, *perm = nullptr;
    uint32_t *sort_scratch = nullptr;   // radix-sort digit counts, scan totals, ping-pong buffers
    int *tile_counter = nullptr;
    __half *Qtc = nullptr;
    unsigned int *qmax_bits = nullptr;
    int tc_mode = 2;              // 0 never, 1 whenever it fits, 2 autotuned
    bool tc_ok = false;
    LaunchPlan plan;
    rift::SkyGrid grid{0, 0};   // sky grid of the current batch size
    // reductions and sampler
    double *red_partial = nullptr, *stats = nullptr, *pooled = nullptr, *final_out = nullptr;
    uint64_t *hist_partial = nullptr;   // [152][6][B][2] exact fixed-point block histograms
    double *pooled_scratch = nullptr;
    uint32_t *sel_idx = nullptr, *sel_count = nullptr;   // RIFT_MIXED re-evaluation list
    double *refine_bins = nullptr;   // RIFT_MIXED: float32 per-bin ln L of the first selected samples
    int64_t refine_rows = 0;
    // large-term correction of the float32 path (k_fixup.cu): the kernels' per-sample
    // template term, largest data term and its bin block; the list of corrected samples;
    // mode-pair tables and double-float copies of U, V, Q
    float *aux_q = nullptr, *aux_m = nullptr;
    int *aux_j = nullptr;
    uint32_t *fix_idx = nullptr, *fix_count = nullptr;
    uint16_t *fix_aij = nullptr, *fix_bij = nullptr;
    int *fix_astart = nullptr, *fix_bstart = nullptr;
    float4 *fix_ua = nullptr, *fix_vb = nullptr, *fix_qdf = nullptr;
    rift::FixTables fix{};
    bool fix_on = false;
    float fix_thr = 0.f;
    double *P = nullptr, *C = nullptr, *Lg = nullptr;
    int *err = nullptr;
    uint32_t *iter_dev = nullptr;   // sampler iteration counter read by the draw kernel
    std::vector<double> host_out;   // err word, pooled record, per-iteration records
    uint32_t iteration = 0;
    int64_t last_n = 0;
    int64_t launches = 0;
    std::vector<std::array<cudaEvent_t, 4>> ev;   // per-iteration stage timers, created on first use
    bool timed = true;        // record the stage timers
    bool capturing = false;   // work is being captured into a graph
    // captured adapt sequence, replayed while its shape repeats
    cudaGraphExec_t graph = nullptr;
    int32_t graph_iter = 0;
    int64_t graph_n = 0;
    LaunchPlan graph_plan;
    int64_t graph_launches = 0;
    int32_t last_shape_iter = 0;   // shape of the previous direct adapt call
    int64_t last_shape_n = 0;
    std::vector<void *> allocs;
    // adaptive-volume integrator state (allocated by the first rift_ile_av call)
    struct AVState {
        int64_t cap = 0;             // live-set capacity
        int level = 0;               // 2^level cells per side
        int64_t n_cells = 1;
        double V = 1.0;              // volume of the active cells
        double V_thr = 1.0;          // estimated volume above the current threshold
        int64_t n_live = 0;
        bool has_thr = false;        // threshold (m, b): keep floor((m - ln L) 64) <= b
        double m = 0.0;
        int64_t b = 0;
        uint32_t iter = 0;
        double *v = nullptr, *lnL = nullptr, *v2 = nullptr, *lnL2 = nullptr;   // live set, ping-pong
        double *v_fresh = nullptr;                                               // [max_samples][6]
        uint64_t *cells = nullptr, *keys = nullptr, *keys_tmp = nullptr;
        uint32_t *flags = nullptr, *scan = nullptr, *sort = nullptr;
        uint64_t *mass_part = nullptr, *mass = nullptr;
        uint32_t *count_part = nullptr, *count = nullptr;
        unsigned long long *maxbits = nullptr;
    } av;
    // portfolio integrator state (allocated by the first rift_ile_portfolio call)
    struct PortfolioState {
        bool alloc = false;
        uint8_t *member = nullptr;              // [max_samples] member that drew each sample
        double *v = nullptr;                    // [max_samples][6] prior-CDF coordinates of the draws
        double *v_av = nullptr, *lnL_av = nullptr;   // the AV member's draws, compacted
        double *part = nullptr;                 // per-member weight sums: block partials
        double *sums = nullptr;                 // [16 + 13 C] the member sums, then the EM sums
        double *gmm_part = nullptr;             // EM sums: block partials
        double *gmm_tab = nullptr;              // the GMM's draw and density table
        uint32_t iter = 0;                      // portfolio iterations since restart
        int32_t members = 0;                    // member bits of the calls since the last restart
        bool have_w = false;
        double W[3] = {0.0, 0.0, 0.0};          // weights of the next batch
        double W_last[3] = {0.0, 0.0, 0.0};
        double n_ess[3] = {0.0, 0.0, 0.0};
        int64_t n_drawn[3] = {0, 0, 0};
        int frozen[3] = {1, 1, 1};
        int active[3] = {0, 0, 0};
        // the Gaussian-mixture member's state (host), C = 0 before it is started
        int gmm_C = 0;
        double gmm_pi[RIFT_GMM_MAX_COMPONENTS] = {};
        double gmm_mu[RIFT_GMM_MAX_COMPONENTS * 6] = {};
        double gmm_sig[RIFT_GMM_MAX_COMPONENTS * 6] = {};
        std::vector<double> gmm_tab_host;      // staging of gmm_tab
    } pf;
};

#define CK(call)                                                                                                        \
    do {                                                                                                                \
        cudaError_t e_ = (call);                                                                                        \
        if (e_ != cudaSuccess) {                                                                                        \
            if (std::getenv("RIFT_ILE_DEBUG"))                                                                          \
                std::fprintf(stderr, "rift_ile: %s at %s:%d: %s\n", #call, __FILE__, __LINE__, cudaGetErrorString(e_)); \
            cudaGetLastError();                                                                                         \
            return RIFT_ECUDA;                                                                                          \
        }                                                                                                               \
    } while (0)

#define RK(call)                 \
    do {                         \
        int r_ = (call);         \
        if (r_ != RIFT_OK)       \
            return r_;           \
    } while (0)

namespace rift {
namespace host {

SamplerDev sampler_of(const rift_ile_t *h);
int map_err(int flags);
bool use_fp32(const rift_ile_t *h);
// Create the stage timers of iteration slots [0, n).
int ensure_events(rift_ile_t *h, int n);
// Enqueue a whole adaptive sequence on h->stream: error reset, n_iter iterations of
// n samples, pooled result (device side only; nothing is read back).
int enqueue_adapt(rift_ile_t *h, int32_t n_iter, int64_t n);
// Read back the error word and the pooled and per-iteration records after the
// enqueued work; synchronises h->stream.
int collect_result(rift_ile_t *h, int n_iter, rift_ile_result *out);
// Fill in h->plan for a batch of n samples: the cached plan of the problem class,
// else (measure) the fastest candidate timed on a batch drawn from the sampler's
// current iteration, else the untuned default.
int choose_plan(rift_ile_t *h, int64_t n, bool measure = true);
bool use_tc(const rift_ile_t *h, int64_t n);
int grid_for_batch(rift_ile_t *h, int64_t n);
cudaError_t launch_tiled(rift_ile_t *h, const double *theta, int64_t n, double *lnL_tmarg, double *lnL_t,
                         const double *lnpw, double *lnw);
void drop_graph(rift_ile_t *h);
int install_overlaps(rift_ile_t *h);
cudaError_t mark(rift_ile_t *h, int slot, int stage);
int refine_batch(rift_ile_t *h, const double *theta, int64_t n, double *lnL_tmarg, const double *lnpw, double *lnw);
int sync_and_err(rift_ile_t *h, int *flags_out = nullptr);
// Device buffer from the stream-ordered pool on the handle's stream, freed at destroy.
template <typename T> int dalloc(rift_ile_t *h, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMallocAsync(&q, count * sizeof(T) + 16, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return RIFT_ENOMEM;
    }
    h->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return RIFT_OK;
}
constexpr int kScratchSlot = RIFT_MAX_ITER;

// Adaptive-volume steps (ile_av.cu) shared with the portfolio integrator.
int av_alloc(rift_ile_t *h, int64_t cap);
int av_restart(rift_ile_t *h);
// Steps 3-5 (live set, threshold, refinement) on n fresh points v [n][6] with their ln L,
// in index order.
int av_update(rift_ile_t *h, const double *v, const double *lnL, int64_t n, double p_thr, int64_t n_min_star);

}  // namespace host
}  // namespace rift
