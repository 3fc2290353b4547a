// r2g_internal.cuh -- shared internals of the sm_103a library: errors, the
// workspace status block, device helpers, and the list-building primitives
// (count scan, stable radix sort, key ranges) that the rasterizer and the
// voxelizer both use.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/r2g.h"

#define R2G_API extern "C" __attribute__((visibility("default")))

namespace r2g {

// ---------------------------------------------------------------- errors

void set_error(const char* fmt, ...);
r2g_status fail(r2g_status s, const char* fmt, ...);
// R2G_E_CUDA with a message if the last launch failed, else R2G_OK.
r2g_status check_launch(const char* what);

// ---------------------------------------------------------------- profiling
// Optional CUDA-event pairs around each hot kernel (or kernel group), enabled by
// r2g_profile_enable; off by default.  Also a count of kernel launches.

enum ProfKernel : int {
    P_PROJECT = 0, P_EMIT, P_SORT, P_RANGES, P_SPLAT_FWD, P_SPLAT_BWD, P_PROJECT_BWD,
    P_VOX_PROJECT, P_VOX_FWD, P_VOX_BWD, P_VOX_CHAIN, P_LOSS, P_TV, P_ADAM, P_VOX_EMIT, P_VOX_SORT,
    P_VOX_RANGES, P_FDK_FILTER, P_FDK_BP, P_INIT_SELECT, P_INIT_KNN, P_METRICS, P_DENSIFY, P_COUNT
};
// The profile ids of one list build's three stages (emission, sorting, ranges).
struct ListProf {
    int emit, sort, ranges;
};
void prof_begin(int k, cudaStream_t s);
void prof_end(int k, cudaStream_t s);
void note_launches(int n);

// ---------------------------------------------------------------- bounded waits

// Polls a device-side wait (the grid barriers of the cooperative list builds) makes
// before it gives up and reports R2G_E_TIMEOUT: r2g_set_wait_limit's value, else
// kGridSyncSpins (polls ~20 ns apart: about 0.1 s).  Read when a launch is issued.
constexpr unsigned long long kGridSyncSpins = 1ull << 22;
unsigned long long wait_polls();

// ---------------------------------------------------------------- workspace

// Status block at offset 0 of every workspace (256 bytes).
struct WsStatus {
    int32_t status;             // R2G_OK, R2G_E_CAPACITY, R2G_E_TIMEOUT or R2G_E_NUMERIC
    int32_t pad;
    unsigned long long needed;  // list entries the last call needed (the most of its view chunks)
    unsigned long long n_keys;  // entries actually emitted = min(needed, capacity)
    unsigned long long pairs;   // gated pairs (counting runs only)
    unsigned long long blocks_done;  // arrival counter of the entry count pass
    unsigned long long grid_sync;    // arrivals at the cooperative list build's grid barriers
    unsigned long long reserved[26];
};
static_assert(sizeof(WsStatus) == 256, "status block is 256 bytes");

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Bump layout over a workspace base pointer.
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    }
};

// ---------------------------------------------------------------- list building

constexpr int kScanBlocks = 148 * 4;     // fixed grid of the count scan and the key emission
constexpr int kSortBlocksMax = 148 * 16; // largest grid of the radix passes
constexpr int kChunk = 128;              // list entries per tile work item
constexpr int kVoxChunk = 32;            // list entries per brick work item
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Scratch the sort needs (block histograms and digit totals), excluding the two
// entry buffers.
size_t sort_scratch_bytes();

// Grid of the radix passes for a given entry capacity (fixed per workspace, so
// the launch sequence does not depend on device data).
int sort_blocks_for(long long capacity);

// Stable LSD radix sort of status->n_keys 64-bit entries (read on the device) by
// bits [32, 32 + key_bits).  Returns the buffer that holds the result (a or b).
uint64_t* radix_sort_u64(uint64_t* a, uint64_t* b, uint32_t* scratch, const WsStatus* status, int key_bits,
                         int sort_blocks, cudaStream_t st);

// Work items: every key's range is cut into chunks of `chunk` entries (kChunk for
// tiles, kVoxChunk for bricks); item = (key << 32) | chunk index; a key's items
// are consecutive.  item_off[key] = index of the key's first item (written for
// non-empty keys); item_status->n_keys = item count.  items must hold
// items_capacity(n_slots, capacity, chunk) entries.
inline long long items_capacity(long long n_slots, long long capacity, int chunk) {
    return n_slots + (capacity + chunk - 1) / chunk + 1;
}
// ranges[k] = [start, end) of key k in the sorted entries (absent keys: [0, 0)), and
// the work items, in one pass over the sorted entries.  item_status must
// directly follow the ranges array in the workspace (one clear covers both).
void build_ranges_items(const uint64_t* sorted, const WsStatus* status, uint2* ranges, int64_t n_slots,
                        WsStatus* item_status, uint32_t* item_off, uint64_t* items, long long items_cap, int chunk,
                        cudaStream_t st);


inline int bits_for(int64_t n_slots) {
    int b = 1;
    while ((int64_t(1) << b) < n_slots) ++b;
    return b;
}

// ---------------------------------------------------------------- internal entry points
// The public calls with device-side selectors for the graph-capturable training
// step: view_sel picks views (and measured projections) by an index read on the
// device; origin_dev overrides grid origins; it_dev supplies Adam's iteration.

r2g_status rasterize_impl(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                          int32_t V, const float* views, const int* view_sel, const r2g_camera* cam,
                          const r2g_raster_opts* opts, float* image, void* ws, size_t ws_bytes, cudaStream_t stream);
// The raster backward in two parts: the per-record moments and the chain rule
// (added to dmean .. drho; with `adam` set, added to adam->grad and the Adam step
// of every Gaussian taken in the same kernel instead, dmean .. drho unused).
struct AdamState;
constexpr int kRasterBwdMoments = 1, kRasterBwdChain = 2;
r2g_status rasterize_backward_impl(int64_t M, const float* mean, const float* scale, const float* quat,
                                   const float* rho, int32_t V, const float* views, const int* view_sel,
                                   const r2g_camera* cam, const r2g_raster_opts* opts, const float* dimage,
                                   float* dmean, float* dscale, float* dquat, float* drho, void* ws, size_t ws_bytes,
                                   cudaStream_t stream, int parts = kRasterBwdMoments | kRasterBwdChain,
                                   const AdamState* adam = nullptr);
r2g_status voxelize_impl(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                         int32_t G, const r2g_grid* grids, const float* origin_dev, float Q3, float* vol, void* ws,
                         size_t ws_bytes, cudaStream_t stream, bool count, bool separate_lists = false);
// The voxel backward in two parts: the per-record moments (dvol -> moments, in the
// workspace) and the chain rule (moments -> gradients, added to dmean .. drho, or
// with kVoxBwdAssign written over them).
constexpr int kVoxBwdMoments = 1, kVoxBwdChain = 2, kVoxBwdAssign = 4;
r2g_status voxelize_backward_impl(int64_t M, const float* mean, const float* scale, const float* quat,
                                  const float* rho, int32_t G, const r2g_grid* grids, float Q3, const float* dvol,
                                  float* dmean, float* dscale, float* dquat, float* drho, void* ws, size_t ws_bytes,
                                  cudaStream_t stream, int parts);
// clear_arrival false: the caller has cleared the arrival counter earlier on the
// stream (projection_loss_clear), so that the SSIM kernel follows the previous
// kernel directly and can take a programmatic dependent launch.
r2g_status projection_loss_impl(int32_t V, int32_t H, int32_t W, const float* render, const float* meas,
                                const int* meas_sel, float lambda_ssim, float* loss, float* drender, void* ws,
                                size_t ws_bytes, cudaStream_t stream, bool clear_arrival = true);
r2g_status projection_loss_clear(int32_t V, int32_t H, int32_t W, void* ws, size_t ws_bytes, cudaStream_t stream);
r2g_status adam_impl(int64_t M, float* raw, float* act, float* grad, float* m, float* v, int32_t it,
                     const int* it_dev, const r2g_adam_opts* opts, cudaStream_t stream);

// ---------------------------------------------------------------- device helpers

// Programmatic dependent launch.  A kernel launched by launch_pdl may become
// resident while the kernel before it on the stream is still running; it calls
// pdl_wait() before its first access to anything earlier kernels wrote (the wait
// returns once they have completed and their writes are visible; without the
// launch attribute it returns at once).  pdl_trigger() lets the next kernel
// launch once every CTA of this one has called it (called at CTA start: the
// dependents then only take resources this grid no longer needs to start).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Hardware approximations, for values that need not match a stated sequence bit for
// bit (1-2 ulp; arguments far from 0 and 2^126): the approximate square root and
// reciprocal instructions.
__device__ __forceinline__ float sqrt_fast(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;

// Block-wide exclusive scan of one uint32 per thread for a 256-thread block.
// Returns the exclusive prefix; *total receives the block sum.  smem holds 8 words.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t* smem, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    uint32_t wsum = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t s = smem[w];
        wsum += (w < warp) ? s : 0u;
        tot += s;
    }
    __syncthreads();
    *total = tot;
    return wsum + x - v;
}

// Block-wide sum of a 64-bit value for a 256-thread block (result valid in all threads).
__device__ __forceinline__ unsigned long long block_sum_u64_256(unsigned long long v, unsigned long long* smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += smem[w];
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------- 3D TV (shared by r2g_tv3d and r2g_tv3d_noalloc)

// Anisotropic 3D TV of G volumes [G][D][D][D] (n = G D^3 voxels) for the 256-thread
// block blockIdx.x: voxel idx's gradient lam inv_cnt (sum of the signs of its
// backward differences minus those of its forward ones) goes to grad[idx]; the
// block's sum of |forward differences| is returned to thread 0.  red: shared [8].
__device__ __forceinline__ float tv3d_block(const float* __restrict__ vol, int D, long long n, float inv_cnt,
                                            float lam, float* __restrict__ grad, float* red) {
    const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
    float part = 0.f;
    if (idx < n) {
        const long long D3 = (long long)D * D * D;
        const long long g = idx / D3;
        const long long l = idx - g * D3;
        const int z = (int)(l / ((long long)D * D)), y = (int)((l / D) % D), x = (int)(l % D);
        const float* vg = vol + g * D3;
        const float c = vg[l];
        float gr = 0.f;
        const long long st[3] = {1, D, (long long)D * D};
        const int co[3] = {x, y, z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (co[a] + 1 < D) {
                const float d = vg[l + st[a]] - c;
                part += fabsf(d);
                gr -= (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f);
            }
            if (co[a] > 0) {
                const float d = c - vg[l - st[a]];
                gr += (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f);
            }
        }
        grad[idx] = lam * inv_cnt * gr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) s += red[w];
    return s;
}

// Sum of n per-block partials p[0..n) in FP64, in a fixed order (a strided sum per
// thread, then a tree), by one 256-thread block; valid in thread 0.  red: shared [256].
__device__ __forceinline__ double sum_partials_256(const float* __restrict__ p, int n, double* red) {
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) s += p[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    return red[0];
}

}  // namespace r2g
