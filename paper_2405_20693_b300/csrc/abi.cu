// abi.cu -- error reporting, workspace status polling and the version string.
#include <stdarg.h>
#include <stdio.h>

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

}  // namespace r2g

using namespace r2g;

R2G_API r2g_status r2g_poll(const void* ws, size_t ws_bytes, r2g_stream stream, int64_t* needed_keys) {
    if (!ws || ws_bytes < sizeof(WsStatus)) return fail(R2G_E_INVAL, "bad workspace");
    WsStatus st;
    if (cudaMemcpyAsync(&st, ws, sizeof(st), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "reading the workspace status failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (needed_keys) *needed_keys = (int64_t)st.needed;
    if (st.status == R2G_E_CAPACITY)
        return fail(R2G_E_CAPACITY, "list entries needed: %llu, capacity: %llu", st.needed, st.n_keys);
    return (r2g_status)st.status;
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
