// abi.cu -- error reporting, workspace status polling and the version string.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "r2g_internal.cuh"

namespace r2g {

static thread_local char g_msg[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
}

r2g_status fail(r2g_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return s;
}

r2g_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(R2G_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return R2G_OK;
}

// ---------------------------------------------------------------- bounded waits

namespace {
std::atomic<unsigned long long> g_wait_polls{0};
}

unsigned long long wait_polls() {
    const unsigned long long p = g_wait_polls.load(std::memory_order_relaxed);
    return p ? p : kGridSyncSpins;
}

// ---------------------------------------------------------------- profiling

namespace {
const char* const kProfNames[P_COUNT] = {"project",    "emit",       "sort",      "ranges",   "splat_fwd",
                                         "splat_bwd",  "project_bwd", "vox_project", "vox_fwd", "vox_bwd",
                                         "vox_chain",  "loss",       "tv",        "adam",    "vox_emit",
                                         "vox_sort",   "vox_ranges", "fdk_filter", "fdk_bp",  "init_select",
                                         "init_knn",   "metrics",    "densify"};
std::atomic<long long> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
uint32_t g_prof_mask = 0xffffffffu;
std::vector<cudaEvent_t> g_events;
size_t g_next = 0;
struct Span {
    size_t a, b;
};
std::vector<Span> g_spans[P_COUNT];
size_t g_open[P_COUNT];
bool g_overflow = false;
}  // namespace

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_begin(int k, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || !((g_prof_mask >> k) & 1u)) return;
    if (g_next + 2 > g_events.size()) {
        g_overflow = true;
        g_open[k] = (size_t)-1;
        return;
    }
    g_open[k] = g_next;
    cudaEventRecord(g_events[g_next++], s);
}

void prof_end(int k, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || !((g_prof_mask >> k) & 1u) || g_open[k] == (size_t)-1) return;
    if (g_next + 1 > g_events.size()) {
        g_overflow = true;
        return;
    }
    cudaEventRecord(g_events[g_next], s);
    g_spans[k].push_back(Span{g_open[k], g_next});
    ++g_next;
    g_open[k] = (size_t)-1;
}

}  // namespace r2g

using namespace r2g;

R2G_API r2g_status r2g_profile_enable(int32_t on, int32_t max_spans) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (on) {
        const size_t want = 2 * (size_t)(max_spans > 0 ? max_spans : 4096);
        while (g_events.size() < want) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return fail(R2G_E_CUDA, "cudaEventCreate failed");
            g_events.push_back(e);
        }
    }
    g_prof_on = on != 0;
    return R2G_OK;
}

R2G_API r2g_status r2g_profile_select(uint32_t kernel_mask) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_mask = kernel_mask;
    return R2G_OK;
}

R2G_API r2g_status r2g_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_next = 0;
    g_overflow = false;
    for (int k = 0; k < P_COUNT; ++k) {
        g_spans[k].clear();
        g_open[k] = (size_t)-1;
    }
    return R2G_OK;
}

R2G_API r2g_status r2g_profile_read(int32_t kernel, int64_t* launches, double* total_ms) {
    if (kernel < 0 || kernel >= P_COUNT || !launches || !total_ms) return fail(R2G_E_INVAL, "bad profile query");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double ms = 0.0;
    for (const Span& sp : g_spans[kernel]) {
        if (cudaEventSynchronize(g_events[sp.b]) != cudaSuccess) return fail(R2G_E_CUDA, "event sync failed");
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g_events[sp.a], g_events[sp.b]) != cudaSuccess)
            return fail(R2G_E_CUDA, "event timing failed");
        ms += t;
    }
    *launches = (int64_t)g_spans[kernel].size();
    *total_ms = ms;
    if (g_overflow) return fail(R2G_E_CAPACITY, "more profiled spans than events; raise max_spans");
    return R2G_OK;
}

R2G_API const char* r2g_profile_name(int32_t kernel) {
    return (kernel >= 0 && kernel < P_COUNT) ? kProfNames[kernel] : "";
}

R2G_API int64_t r2g_launch_count(void) { return g_launches.load(); }

R2G_API r2g_status r2g_poll(const void* ws, size_t ws_bytes, r2g_stream stream, int64_t* needed_keys) {
    if (!ws || ws_bytes < sizeof(WsStatus)) return fail(R2G_E_INVAL, "bad workspace");
    WsStatus st;
    if (cudaMemcpyAsync(&st, ws, sizeof(st), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "reading the workspace status failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (needed_keys) *needed_keys = (int64_t)st.needed;
    if (st.status == R2G_E_CAPACITY)
        return fail(R2G_E_CAPACITY, "list entries needed: %llu, capacity: %llu", st.needed, st.n_keys);
    if (st.status == R2G_E_TIMEOUT)
        return fail(R2G_E_TIMEOUT, "a grid barrier of the list build gave up after %llu polls", wait_polls());
    if (st.status == R2G_E_NUMERIC)
        return fail(R2G_E_NUMERIC, "a non-finite loss: the step left the parameters and moments unchanged");
    return (r2g_status)st.status;
}

R2G_API r2g_status r2g_set_wait_limit(uint64_t polls) {
    g_wait_polls.store(polls, std::memory_order_relaxed);
    return R2G_OK;
}

R2G_API r2g_status r2g_pair_count(const void* ws, size_t ws_bytes, int64_t* pairs, r2g_stream stream) {
    if (!ws || !pairs || ws_bytes < sizeof(WsStatus)) return fail(R2G_E_INVAL, "bad workspace or NULL pointer");
    WsStatus st;
    if (cudaMemcpyAsync(&st, ws, sizeof(st), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "reading the workspace status failed");
    *pairs = (int64_t)st.pairs;
    return R2G_OK;
}

R2G_API const char* r2g_last_error(void) { return g_msg; }

R2G_API const char* r2g_version(void) { return "r2g 0.1 (sm_103a)"; }
