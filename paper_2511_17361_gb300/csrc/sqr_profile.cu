// sqr_profile.cu -- optional per-kernel timing of the library's launches.
//
// While enabled, prof_begin / prof_end record a CUDA event on the launching
// stream before and after every kernel launch of the library, tagged with the
// kernel's name.  sq_profile_query waits for the events and sums the durations
// per name.  Disabled (the default) the two calls return at once.
#include <atomic>
#include <mutex>
#include <string.h>
#include <vector>

#include "sqr_common.cuh"

namespace sqr {

namespace {

struct Record {
    const char* name;  // string literal of the launch site
    int ev;            // index of the begin event; ev + 1 is the end event
};

std::mutex g_mu;
std::atomic<bool> g_on{false};
std::vector<cudaEvent_t> g_events;  // pairs, created on demand
std::vector<Record> g_records;
long long g_dropped = 0;
thread_local int t_open = -1;  // begin event of this thread's launch in progress

}  // namespace

void prof_begin(const char* name, cudaStream_t st) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    t_open = -1;
    if ((long long)g_records.size() >= SQ_PROFILE_MAX_LAUNCHES) {
        ++g_dropped;
        return;
    }
    const int ev = (int)g_records.size() * 2;
    while ((int)g_events.size() < ev + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            ++g_dropped;
            return;
        }
        g_events.push_back(e);
    }
    if (cudaEventRecord(g_events[ev], st) != cudaSuccess) {
        ++g_dropped;
        return;
    }
    g_records.push_back(Record{name, ev});
    t_open = ev;
}

void prof_end(cudaStream_t st) {
    if (t_open < 0) return;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaEventRecord(g_events[t_open + 1], st);
    t_open = -1;
}

}  // namespace sqr

extern "C" sq_status_t sq_profile_enable(int on) {
    using namespace sqr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (on) {
        g_records.clear();
        g_dropped = 0;
    }
    g_on.store(on != 0);
    return SQ_OK;
}

extern "C" sq_status_t sq_profile_query(const char* name, long long* launches, double* total_ms, long long* dropped) {
    using namespace sqr;
    if (!launches || !total_ms) {
        set_last_error("sq_profile_query: NULL output");
        return SQ_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    long long n = 0;
    double ms = 0.0;
    for (const Record& r : g_records) {
        if (name && strcmp(name, r.name) != 0) continue;
        cudaError_t e = cudaEventSynchronize(g_events[r.ev + 1]);
        if (e != cudaSuccess) return cuda_status(e, "sq_profile_query: event");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, g_events[r.ev], g_events[r.ev + 1]);
        if (e != cudaSuccess) return cuda_status(e, "sq_profile_query: elapsed time");
        ++n;
        ms += t;
    }
    *launches = n;
    *total_ms = ms;
    if (dropped) *dropped = g_dropped;
    return SQ_OK;
}
