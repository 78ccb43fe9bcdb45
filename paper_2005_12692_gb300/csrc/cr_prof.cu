// cr_prof.cu -- launch accounting and optional per-stage timing with CUDA
// events recorded on the caller's stream (diagnostics for benchmarks; off
// by default, in which case a stage marker costs one branch).
#include "cr_internal.cuh"
#include <atomic>
#include <mutex>
#include <vector>

namespace cr {

std::atomic<long long> g_launch_count{0};

static const char *kStageNames[STAGE_COUNT] = {
    "h0_stencil", "jump",        "roots",      "relabel",    "h0_cross",   "uf_round",
    "dual_stencil", "dual_cross", "h1_scan",   "h1_sort",    "h1_reduce",  "h1_emit",
    "out_sort",   "bw_contrib",  "bw_sort",    "bw_sum",     "images",     "h1_columns"};

struct Pending {
    int stage;
    cudaEvent_t a, b;
    double bytes;
    bool graph_owned;  // recorded by a graph node: re-used by every launch of the graph
};

static std::mutex g_mu;
static bool g_on = false;
static uint32_t g_mask = 0xFFFFFFFFu;  // stages that record events
static std::vector<cudaEvent_t> g_pool;
static std::vector<Pending> g_pending;
static std::vector<Pending> g_open;  // begun, not ended
static bool g_capturing = false;    // a stream capture is recording the stages
static std::vector<Pending> g_captured;
static double g_ms[STAGE_COUNT];
static long long g_n[STAGE_COUNT];
static double g_bytes[STAGE_COUNT];

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(cudaStream_t st, int stage) {
    if (!g_on || !((g_mask >> stage) & 1u)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Pending p{stage, take_event(), nullptr, 0.0, g_capturing};
    if (g_capturing)
        cudaEventRecordWithFlags(p.a, st, cudaEventRecordExternal);  // a timing node of the graph
    else
        cudaEventRecord(p.a, st);
    g_open.push_back(p);
}

void prof_end(cudaStream_t st, int stage, double bytes) {
    if (!g_on || !((g_mask >> stage) & 1u)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = g_open.size(); i-- > 0;) {
        if (g_open[i].stage == stage) {
            Pending p = g_open[i];
            g_open.erase(g_open.begin() + (long)i);
            p.b = take_event();
            p.bytes = bytes;
            if (p.graph_owned) {
                cudaEventRecordWithFlags(p.b, st, cudaEventRecordExternal);
                g_captured.push_back(p);
            } else {
                cudaEventRecord(p.b, st);
                g_pending.push_back(p);
            }
            return;
        }
    }
}

// bytes known only after the stream reached this point (device counters)
void prof_add_bytes(int stage, double bytes) {
    if (!g_on || !((g_mask >> stage) & 1u)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_bytes[stage] += bytes;
}

void prof_flush() {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.stage] += ms;
            g_n[p.stage] += 1;
            g_bytes[p.stage] += p.bytes;
        }
        if (!p.graph_owned) {
            g_pool.push_back(p.a);
            g_pool.push_back(p.b);
        }
    }
    g_pending.clear();
}

bool prof_active() { return g_on; }
uint32_t prof_mask() { return g_mask; }

// stages recorded while a graph is captured become event nodes of the graph;
// their events belong to the graph and are read after every launch of it
void prof_capture_begin() {
    std::lock_guard<std::mutex> lk(g_mu);
    g_capturing = true;
    g_captured.clear();
}
void prof_capture_end(std::vector<std::pair<int, std::pair<void *, void *>>> &out, std::vector<double> &bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_capturing = false;
    out.clear();
    bytes.clear();
    for (auto &p : g_captured) {
        out.push_back({p.stage, {(void *)p.a, (void *)p.b}});
        bytes.push_back(p.bytes);
    }
    g_captured.clear();
}
void prof_replay(const std::vector<std::pair<int, std::pair<void *, void *>>> &recs, const std::vector<double> &bytes) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < recs.size(); i++)
        g_pending.push_back(Pending{recs[i].first, (cudaEvent_t)recs[i].second.first,
                                    (cudaEvent_t)recs[i].second.second, bytes[i], true});
}

}  // namespace cr

extern "C" {

int cr_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(cr::g_mu);
    cr::g_on = on != 0;
    return CR_OK;
}

int cr_profile_select(uint32_t stage_mask) {
    std::lock_guard<std::mutex> lk(cr::g_mu);
    cr::g_mask = stage_mask;
    return CR_OK;
}

void cr_profile_reset(void) {
    std::lock_guard<std::mutex> lk(cr::g_mu);
    for (int i = 0; i < cr::STAGE_COUNT; i++) {
        cr::g_ms[i] = 0;
        cr::g_n[i] = 0;
        cr::g_bytes[i] = 0;
    }
}

int cr_profile_read(int stage, const char **name, double *total_ms, int64_t *count, double *bytes) {
    if (stage < 0 || stage >= cr::STAGE_COUNT) return CR_ERR_INVALID_ARG;
    cr::prof_flush();
    std::lock_guard<std::mutex> lk(cr::g_mu);
    if (name) *name = cr::kStageNames[stage];
    if (total_ms) *total_ms = cr::g_ms[stage];
    if (count) *count = cr::g_n[stage];
    if (bytes) *bytes = cr::g_bytes[stage];
    return CR_OK;
}

int64_t cr_launch_count(void) { return (int64_t)cr::g_launch_count.load(); }

}  // extern "C"
