// tv_noalloc.cu -- r2g_tv3d_noalloc: the 3D TV loss and gradient with no
// caller-provided workspace and no allocation anywhere.
//
// Who needs this: code that may not allocate device memory at the point it runs
// -- for example a host application that hands this library a fixed device
// budget up front and forbids cudaMalloc afterwards, a real-time loop in which an
// allocation (or a caching allocator's fallback to cudaMalloc) would stall, or
// a plugin that only ever receives input and output buffers from its host.
// Those callers cannot size and pass the per-block partial-sum workspace that
// r2g_tv3d takes, so this variant keeps that scratch in a fixed device array
// that is part of the library image.
//
// The array (kTvStaticPartials floats = 256 KiB) lives on every device that
// loads the library until the process exits.  Its host-side name is only a
// stand-in: host code must not pass it to a kernel.  The first call on each
// device (with that device current) looks up the array's device address with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture.  The cached address belongs to the device's primary context: a
// cudaDeviceReset, or a call from a different (non-primary) context on the same
// device, may load the module again at another address, and the cached one is
// then stale -- such callers must not use this entry point after the change.  All
// calls share the one array, which keeps the last call's contents; every block
// overwrites its own partial before the final sum reads it, so nothing has to be
// cleared between calls.  Calls whose kernels overlap on the GPU (different
// streams, no ordering) race on the array.
#include <math.h>

#include <mutex>

#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr long long kTvStaticPartials = 65536;  // one float per 256-voxel block: up to 2^24 voxels

static __device__ __align__(256) float g_tv_partials[kTvStaticPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_addr[kMaxDevices] = {nullptr};

// The workspace-based TV kernels' own per-voxel and per-block arithmetic and their
// fixed-order final sum (tv3d_block, sum_partials_256), with the partials in the
// fixed array: the same loss and gradient as r2g_tv3d, bit for bit.
__global__ void __launch_bounds__(256) k_tv3d_static(const float* __restrict__ vol, int D, long long n,
                                                     float inv_cnt, float lam, float* __restrict__ grad,
                                                     float* __restrict__ partials) {
    __shared__ float red[8];
    const float s = tv3d_block(vol, D, n, inv_cnt, lam, grad, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_tv_sum_static(const float* __restrict__ p, int n, float scale,
                                                       float* __restrict__ loss) {
    __shared__ double red[256];
    const double s = sum_partials_256(p, n, red);
    if (threadIdx.x == 0) *loss = (float)(scale * s);
}

// Device address of the static array on the current device (looked up once per device).
r2g_status static_partials(float** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(R2G_E_CUDA, "r2g_tv3d_noalloc: no usable current CUDA device");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_tv_partials);
        if (e != cudaSuccess || !p)
            return fail(R2G_E_CUDA, "r2g_tv3d_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                        cudaGetErrorString(e));
        g_addr[dev] = static_cast<float*>(p);
    }
    *out = g_addr[dev];
    return R2G_OK;
}

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API r2g_status r2g_tv3d_noalloc(int32_t G, int32_t D, const float* vol, float lambda_tv, float* loss,
                                    float* dvol, r2g_stream stream) {
    if (G < 1 || D < 2 || D > 1024) return fail(R2G_E_INVAL, "r2g_tv3d_noalloc: bad volume shape G=%d D=%d", G, D);
    if (!vol || !loss || !dvol) return fail(R2G_E_INVAL, "r2g_tv3d_noalloc: NULL pointer");
    const long long n = (long long)G * D * D * D;
    const long long blocks = (n + 255) / 256;
    if (blocks > kTvStaticPartials)
        return fail(R2G_E_INVAL,
                    "r2g_tv3d_noalloc: %lld voxels exceed the fixed scratch (at most %lld voxels, i.e. "
                    "G * D^3 <= 16777216); use r2g_tv3d with a workspace",
                    n, kTvStaticPartials * 256);
    float* partials = nullptr;
    r2g_status e = static_partials(&partials);
    if (e) return e;
    const float inv_cnt = (float)(1.0 / ((double)D * D * (D - 1)));
    k_tv3d_static<<<(unsigned)blocks, 256, 0, stream>>>(vol, D, n, inv_cnt, lambda_tv, dvol, partials);
    k_tv_sum_static<<<1, 256, 0, stream>>>(partials, (int)blocks, lambda_tv * inv_cnt, loss);
    note_launches(2);
    return check_launch("r2g_tv3d_noalloc");
}
