// Optional per-stage timing for benchmarks: when enabled, selected launches
// are bracketed by CUDA events recorded on their own stream; the elapsed
// times are summed per stage kind on request.  Off by default (no events).
#include "internal.cuh"
#include "timing.cuh"

#include <mutex>
#include <vector>

namespace rpca {

namespace {

struct Rec { int kind; cudaEvent_t a, b; };

std::mutex g_mu;
bool g_on = false;
uint32_t g_mask = 0xffffffffu;     // kinds that record events
std::vector<Rec> g_recs;       // recorded in the current window
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// A stream being captured into a CUDA graph turns a plain event record into a
// dependency edge; an external record becomes an event node that every replay records.
void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

}  // namespace

bool timing_on() { return g_on; }

TimedScope::TimedScope(int kind, cudaStream_t s) : kind_(kind), s_(s) {
    if (!g_on || kind < 0 || kind > 31 || !((g_mask >> kind) & 1u)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    b_ = take_event();
    if (a_) record(a_, s_);
}

TimedScope::~TimedScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (b_) record(b_, s_);
    g_recs.push_back({kind_, a_, b_});
}

}  // namespace rpca

extern "C" int rpca_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(rpca::g_mu);
    rpca::g_on = on != 0;
    // on > 1: create that many events now, outside the window being timed
    for (int32_t i = (int32_t)rpca::g_pool.size(); i < on; ++i) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return RPCA_ERR_CUDA;
        rpca::g_pool.push_back(e);
    }
    return RPCA_OK;
}

extern "C" int rpca_timing_select(uint32_t kinds_mask) {
    std::lock_guard<std::mutex> lk(rpca::g_mu);
    rpca::g_mask = kinds_mask;
    return RPCA_OK;
}

extern "C" int rpca_timing_reset(void) {
    std::lock_guard<std::mutex> lk(rpca::g_mu);
    for (auto &r : rpca::g_recs) { rpca::g_pool.push_back(r.a); rpca::g_pool.push_back(r.b); }
    rpca::g_recs.clear();
    return RPCA_OK;
}

extern "C" int rpca_timing_read(int32_t kind, int64_t *count, double *total_ms) {
    if (!count || !total_ms) return RPCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(rpca::g_mu);
    int64_t c = 0;
    double t = 0.0;
    for (auto &r : rpca::g_recs) {
        if (r.kind != kind) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return RPCA_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return RPCA_ERR_CUDA;
        ++c;
        t += ms;
    }
    *count = c;
    *total_ms = t;
    return RPCA_OK;
}
