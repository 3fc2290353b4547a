// emit.cuh -- count, scan and emit of (key, Gaussian id) list entries, shared by
// the rasterizer (key = tile) and the voxelizer (key = brick).
//
// An Op supplies, for record r, how many entries it emits (count) and writes them
// (emit).  Records are split into kScanBlocks contiguous chunks; a first pass sums
// each chunk, one block scans the chunk sums (and writes the total and the
// capacity verdict into the status block), and a second pass re-scans each chunk
// in rounds of 256 records and writes every record's entries at its offset, in
// record order.  Entries beyond the capacity are not written.
#pragma once

#include "r2g_internal.cuh"

namespace r2g {

template <class Op>
__global__ void __launch_bounds__(256) k_count_chunks(Op op, long long n_rec, unsigned long long* partials) {
    __shared__ unsigned long long sm[8];
    const long long chunk = (n_rec + gridDim.x - 1) / gridDim.x;
    const long long begin = min(n_rec, (long long)blockIdx.x * chunk);
    const long long end = min(n_rec, begin + chunk);
    unsigned long long s = 0;
    for (long long r = begin + threadIdx.x; r < end; r += 256) s += op.count(r);
    s = block_sum_u64_256(s, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One block of 1024 threads; nb <= 1024.  partials become exclusive offsets.
static __global__ void __launch_bounds__(1024) k_scan_chunks(unsigned long long* partials, int nb, WsStatus* st,
                                                      unsigned long long capacity) {
    __shared__ unsigned long long wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long v = tid < nb ? partials[tid] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;  // inclusive
    }
    __syncthreads();
    const unsigned long long before = (warp > 0 ? wsum[warp - 1] : 0ull) + x - v;
    if (tid < nb) partials[tid] = before;
    if (tid == 0) {
        const unsigned long long total = wsum[31];
        st->needed = total;
        st->n_keys = total < capacity ? total : capacity;
        if (total > capacity) st->status = R2G_E_CAPACITY;
    }
}

template <class Op>
__global__ void __launch_bounds__(256) k_emit_chunks(Op op, long long n_rec, const unsigned long long* partials,
                                                     uint64_t* out, unsigned long long capacity) {
    __shared__ uint32_t sm[8];
    const long long chunk = (n_rec + gridDim.x - 1) / gridDim.x;
    const long long begin = min(n_rec, (long long)blockIdx.x * chunk);
    const long long end = min(n_rec, begin + chunk);
    unsigned long long running = partials[blockIdx.x];
    for (long long base = begin; base < end; base += 256) {
        const long long r = base + threadIdx.x;
        const uint32_t c = r < end ? op.count(r) : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(c, sm, &tot);
        if (c) op.emit(r, out, running + ex, capacity);
        running += tot;
    }
}

// Launch the three steps; the status block must have been cleared by the caller.
template <class Op>
void emit_lists(const Op& op, long long n_rec, unsigned long long* partials, WsStatus* st, uint64_t* out,
                unsigned long long capacity, cudaStream_t s) {
    k_count_chunks<Op><<<kScanBlocks, 256, 0, s>>>(op, n_rec, partials);
    k_scan_chunks<<<1, 1024, 0, s>>>(partials, kScanBlocks, st, capacity);
    k_emit_chunks<Op><<<kScanBlocks, 256, 0, s>>>(op, n_rec, partials, out, capacity);
}

}  // namespace r2g
