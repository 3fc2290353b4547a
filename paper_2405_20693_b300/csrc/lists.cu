// lists.cu -- the sort and range primitives behind the per-tile and per-brick
// Gaussian lists: a stable LSD radix sort of 64-bit entries (key in the upper
// 32 bits, Gaussian id in the lower 32) and the [start, end) range of each key.
//
// The sort is reduce-then-scan with a FIXED grid: the entry count is produced
// on the device by the key emission and read here from the workspace status, so
// no host round trip is needed and the whole call sequence can be captured in a
// CUDA graph.  Each pass: per-block digit histograms, per-digit offsets, and a
// scatter in which each 256-element round is ranked with warp match masks so
// the order of equal digits is kept (stability makes every per-key list come out
// in ascending Gaussian id).
#include "r2g_internal.cuh"

namespace r2g {

namespace {

constexpr int kMaxPasses = 4;

__device__ __forceinline__ void chunk_of(unsigned long long n, unsigned long long& begin, unsigned long long& end) {
    const unsigned long long chunk = (n + gridDim.x - 1) / gridDim.x;
    begin = min(n, (unsigned long long)blockIdx.x * chunk);
    end = min(n, begin + chunk);
}

__global__ void __launch_bounds__(256) k_radix_hist(const uint64_t* __restrict__ in, const WsStatus* __restrict__ st,
                                                    uint32_t* __restrict__ hist, uint32_t* __restrict__ digit_total,
                                                    int shift, uint32_t mask) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long begin, end;
    chunk_of(st->n_keys, begin, end);
    for (unsigned long long i = begin + threadIdx.x; i < end; i += 256) {
        const uint32_t d = (uint32_t)(in[i] >> shift) & mask;
        atomicAdd(&h[d], 1u);
    }
    __syncthreads();
    const uint32_t c = h[threadIdx.x];
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = c;
    if (c) atomicAdd(&digit_total[threadIdx.x], c);
}

// One block per digit: offset of (digit, block) = entries of smaller digits +
// entries of this digit in earlier blocks.  Overwrites hist in place.
__global__ void __launch_bounds__(1024) k_radix_offsets(uint32_t* __restrict__ hist,
                                                        const uint32_t* __restrict__ digit_total, int nblocks) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_base;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        uint32_t part = 0;
        for (int k = lane; k < d; k += 32) part += digit_total[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_base = part;
    }
    __syncthreads();
    uint32_t running = s_base;
    uint32_t* row = hist + (size_t)d * nblocks;
    for (int c = 0; c < nblocks; c += 1024) {
        const int idx = c + tid;
        const uint32_t v = idx < nblocks ? row[idx] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? wsum[warp - 1] : 0u) + x - v;
        if (idx < nblocks) row[idx] = running + before;
        running += wsum[31];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_radix_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                       const uint32_t* __restrict__ offs,
                                                       const WsStatus* __restrict__ st, int shift, uint32_t mask) {
    __shared__ uint32_t s_run[kRadix];
    __shared__ uint32_t s_cnt[8][kRadix];
    __shared__ uint32_t s_tot[kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_run[tid] = offs[(size_t)tid * gridDim.x + blockIdx.x];
#pragma unroll
    for (int w = 0; w < 8; ++w) s_cnt[w][tid] = 0;
    __syncthreads();
    unsigned long long begin, end;
    chunk_of(st->n_keys, begin, end);
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (unsigned long long base = begin; base < end; base += 256) {
        const unsigned long long idx = base + tid;
        const bool valid = idx < end;
        const uint64_t x = valid ? in[idx] : 0ull;
        const uint32_t d = valid ? ((uint32_t)(x >> shift) & mask) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const uint32_t c = s_cnt[w][tid];
                s_cnt[w][tid] = acc;
                acc += c;
            }
            s_tot[tid] = acc;
        }
        __syncthreads();
        if (valid) out[s_run[d] + s_cnt[warp][d] + rank] = x;
        __syncthreads();
        s_run[tid] += s_tot[tid];
#pragma unroll
        for (int w = 0; w < 8; ++w) s_cnt[w][tid] = 0;
        __syncthreads();
    }
}

}  // namespace

size_t sort_scratch_bytes() {
    return ((size_t)kRadix * kSortBlocksMax + (size_t)kRadix * kMaxPasses) * sizeof(uint32_t);
}

int sort_blocks_for(long long capacity) {
    long long nb = (capacity + 4095) / 4096;  // about 4096 entries (16 rounds) per block when full
    if (nb < 148) nb = 148;
    if (nb > kSortBlocksMax) nb = kSortBlocksMax;
    return (int)nb;
}

uint64_t* radix_sort_u64(uint64_t* a, uint64_t* b, uint32_t* scratch, const WsStatus* status, int key_bits,
                         int nb, cudaStream_t st) {
    if (key_bits < 1) key_bits = 1;
    if (key_bits > 32) key_bits = 32;
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    const int bpp = (key_bits + passes - 1) / passes;
    uint32_t* hist = scratch;
    uint32_t* totals = scratch + (size_t)kRadix * kSortBlocksMax;
    cudaMemsetAsync(totals, 0, sizeof(uint32_t) * kRadix * kMaxPasses, st);
    uint64_t* src = a;
    uint64_t* dst = b;
    for (int p = 0; p < passes; ++p) {
        const int shift = 32 + p * bpp;
        const uint32_t mask = (1u << bpp) - 1u;
        uint32_t* tot = totals + (size_t)kRadix * p;
        k_radix_hist<<<nb, 256, 0, st>>>(src, status, hist, tot, shift, mask);
        k_radix_offsets<<<1u << bpp, 1024, 0, st>>>(hist, tot, nb);
        k_radix_scatter<<<nb, 256, 0, st>>>(src, dst, hist, status, shift, mask);
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

namespace {

// At the first entry of every key: find the key's end by binary search, write its
// range, and claim ceil(n / chunk) consecutive work items with one atomic.  The
// order in which keys claim their items varies from run to run, but each key's
// items are contiguous and numbered by chunk, so every consumer that combines a
// key's chunks does so in chunk order.
__global__ void __launch_bounds__(256) k_ranges_items(const uint64_t* __restrict__ s,
                                                      const WsStatus* __restrict__ st, uint2* __restrict__ ranges,
                                                      unsigned long long n_slots, WsStatus* __restrict__ item_st,
                                                      uint32_t* __restrict__ item_off, uint64_t* __restrict__ items,
                                                      unsigned long long items_cap, uint32_t chunk) {
    const unsigned long long n = st->n_keys;
    for (unsigned long long i = (unsigned long long)blockIdx.x * 256 + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * 256) {
        const uint32_t k = (uint32_t)(s[i] >> 32);
        if (k >= n_slots) continue;
        if (i != 0 && (uint32_t)(s[i - 1] >> 32) == k) continue;
        unsigned long long lo = i + 1, hi = n;  // first index whose key differs
        while (lo < hi) {
            const unsigned long long mid = (lo + hi) >> 1;
            if ((uint32_t)(s[mid] >> 32) == k) lo = mid + 1;
            else hi = mid;
        }
        ranges[k] = make_uint2((uint32_t)i, (uint32_t)lo);
        const uint32_t nch = (uint32_t)((lo - i + chunk - 1) / chunk);
        const unsigned long long base = atomicAdd(&item_st->n_keys, (unsigned long long)nch);
        item_off[k] = (uint32_t)base;
        for (uint32_t c = 0; c < nch; ++c)
            if (base + c < items_cap) items[base + c] = ((uint64_t)k << 32) | c;
    }
}

}  // namespace

void build_ranges_items(const uint64_t* sorted, const WsStatus* status, uint2* ranges, int64_t n_slots,
                        WsStatus* item_status, uint32_t* item_off, uint64_t* items, long long items_cap, int chunk,
                        cudaStream_t st) {
    // ranges and the item status block are adjacent in every workspace: one clear
    cudaMemsetAsync(ranges, 0, reinterpret_cast<char*>(item_status) - reinterpret_cast<char*>(ranges) +
                                   sizeof(WsStatus), st);
    k_ranges_items<<<148 * 8, 256, 0, st>>>(sorted, status, ranges, (unsigned long long)n_slots, item_status,
                                            item_off, items, (unsigned long long)items_cap, (uint32_t)chunk);
}

}  // namespace r2g
