// emit.cuh -- count, scan and emit of (key, Gaussian id) list entries, shared by
// the rasterizer (key = tile) and the voxelizer (key = brick), and the list
// builder that turns them into per-key lists sorted by Gaussian id.
//
// An Op supplies, for record r, how many entries it emits (count) and visits them
// in order (entries(r, f) calls f(key, id) once per entry).  Records are split
// into contiguous chunks, one per block; a first pass sums each chunk (its last
// block to finish scans the chunk sums and writes the total and the capacity
// verdict into the status block), and a second pass re-scans each chunk in
// rounds of 256 records and writes every record's entries at its offset, in
// record order.  Entries beyond the capacity are not written.
//
// Key spaces of at most kFusedKeys keys (one 512^2 view in 16 x 16 tiles, the
// bricks of a TV patch) take a fused path: the emission also counts its block's
// entries per key, one warp per key turns the counts into scatter offsets, the
// key's range and its work items, and a stable scatter (one contiguous run per
// warp, ranked with warp match masks) writes the sorted lists -- four launches
// and one pass over the entries.  Larger key spaces take the general stable LSD
// radix sort and a range pass.
#pragma once

#include "r2g_internal.cuh"

namespace r2g {

constexpr int kFusedKeys = 1024;
constexpr int kFusedBlocks = 148;  // emit / scatter blocks of the fused path
static_assert(kScanBlocks <= 1024 && kFusedBlocks <= 1024, "the last count block scans <= 1024 chunk sums");
static_assert((size_t)kFusedKeys * kFusedBlocks <= (size_t)kRadix * kSortBlocksMax,
              "fused histograms fit the sort scratch");
static_assert(kFusedKeys <= kRadix * 4, "fused key totals fit the sort scratch");

// Block-wide exclusive scan of a 64-bit value for a 256-thread block.
__device__ __forceinline__ unsigned long long block_excl_scan_u64_256(unsigned long long v, unsigned long long* smem,
                                                                      unsigned long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    unsigned long long before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const unsigned long long t = smem[w];
        before += (w < warp) ? t : 0ull;
        tot += t;
    }
    __syncthreads();
    *total = tot;
    return before + x - v;
}

// Each block sums the entry counts of its contiguous chunk of records.  The last
// block to finish (arrival counter in the status block, cleared by the caller)
// turns the gridDim.x <= 1024 chunk sums into exclusive offsets, writes the total
// and the capacity verdict, and clears key_totals (fused path) for the emission.
template <class Op>
__global__ void __launch_bounds__(256) k_count_chunks(Op op, long long n_rec, unsigned long long* partials,
                                                      WsStatus* st, unsigned long long capacity,
                                                      uint32_t* key_totals, int n_keys) {
    __shared__ unsigned long long sm[8];
    __shared__ int s_last;
    const long long chunk = (n_rec + gridDim.x - 1) / gridDim.x;
    const long long begin = min(n_rec, (long long)blockIdx.x * chunk);
    const long long end = min(n_rec, begin + chunk);
    unsigned long long s = 0;
    for (long long r = begin + threadIdx.x; r < end; r += 256) s += op.count(r);
    s = block_sum_u64_256(s, sm);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        s_last = atomicAdd(&st->blocks_done, 1ull) == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nb = (int)gridDim.x, t = threadIdx.x;
    unsigned long long v[4], mine = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 4 * t + q;
        v[q] = i < nb ? __ldcg(partials + i) : 0ull;
        mine += v[q];
    }
    unsigned long long total;
    unsigned long long run = block_excl_scan_u64_256(mine, sm, &total);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 4 * t + q;
        if (i < nb) partials[i] = run;
        run += v[q];
    }
    if (key_totals)
        for (int k = t; k < n_keys; k += 256) key_totals[k] = 0;
    if (t == 0) {
        st->needed = total;
        st->n_keys = total < capacity ? total : capacity;
        if (total > capacity) st->status = R2G_E_CAPACITY;
    }
}

// HIST (fused path): also count the block's written entries per key, then store
// the counts as hist[key * gridDim.x + block] and add them to key_totals.
template <class Op, bool HIST>
__global__ void __launch_bounds__(256) k_emit_chunks(Op op, long long n_rec, const unsigned long long* partials,
                                                     uint64_t* out, unsigned long long capacity,
                                                     uint32_t* __restrict__ hist, uint32_t* __restrict__ key_totals,
                                                     int n_keys) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t h[HIST ? kFusedKeys : 1];
    if (HIST) {
        for (int k = threadIdx.x; k < n_keys; k += 256) h[k] = 0;
        __syncthreads();
    }
    const long long chunk = (n_rec + gridDim.x - 1) / gridDim.x;
    const long long begin = min(n_rec, (long long)blockIdx.x * chunk);
    const long long end = min(n_rec, begin + chunk);
    unsigned long long running = partials[blockIdx.x];
    for (long long base = begin; base < end; base += 256) {
        const long long r = base + threadIdx.x;
        const uint32_t c = r < end ? op.count(r) : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(c, sm, &tot);
        if (c) {
            unsigned long long off = running + ex;
            op.entries(r, [&](uint32_t key, uint32_t id) {
                if (off < capacity) {
                    out[off] = ((uint64_t)key << 32) | (uint64_t)id;
                    if (HIST) atomicAdd(&h[key], 1u);
                }
                ++off;
            });
        }
        running += tot;
    }
    if (HIST) {
        __syncthreads();
        for (int k = threadIdx.x; k < n_keys; k += 256) {
            const uint32_t cnt = h[k];
            hist[(size_t)k * gridDim.x + blockIdx.x] = cnt;
            if (cnt) atomicAdd(&key_totals[k], cnt);
        }
    }
}

// One warp per key k: the scatter offset of (k, emit block b) = entries of
// smaller keys + entries of key k in earlier blocks (hist rewritten in place),
// the key's range [start, end) ([0, 0) when empty), its first work item and its
// max(1, ceil(n / chunk)) items (an empty key's one item writes its zero output),
// a cleared chunk arrival counter; the last key's warp writes the item count.
static __global__ void __launch_bounds__(256) k_fused_offsets(uint32_t* __restrict__ hist,
                                                              const uint32_t* __restrict__ key_totals, int nb,
                                                              int n_keys, uint32_t chunk, uint2* __restrict__ ranges,
                                                              uint32_t* __restrict__ key_done,
                                                              uint32_t* __restrict__ item_off,
                                                              uint64_t* __restrict__ items,
                                                              unsigned long long items_cap,
                                                              WsStatus* __restrict__ item_st) {
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= n_keys) return;
    uint32_t base = 0, ibase = 0;
    for (int q = lane; q < k; q += 32) {
        const uint32_t t = key_totals[q];
        base += t;
        ibase += t ? (t + chunk - 1) / chunk : 1u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        base += __shfl_xor_sync(0xffffffffu, base, o);
        ibase += __shfl_xor_sync(0xffffffffu, ibase, o);
    }
    uint32_t running = base;
    uint32_t* row = hist + (size_t)k * nb;
    for (int c = 0; c < nb; c += 32) {
        const int idx = c + lane;
        const uint32_t v = idx < nb ? row[idx] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (idx < nb) row[idx] = running + x - v;
        running += __shfl_sync(0xffffffffu, x, 31);
    }
    const uint32_t total = key_totals[k];
    const uint32_t nch = total ? (total + chunk - 1) / chunk : 1u;
    if (lane == 0) {
        ranges[k] = total ? make_uint2(base, base + total) : make_uint2(0u, 0u);
        key_done[k] = 0;
        item_off[k] = ibase;
        if (k == n_keys - 1) item_st->n_keys = (unsigned long long)ibase + nch;
    }
    for (uint32_t c = lane; c < nch; c += 32)
        if (ibase + c < items_cap) items[ibase + c] = ((uint64_t)(uint32_t)k << 32) | c;
}

// One block per emit block: its entries [start_b, start_{b+1}) (clipped to the
// written count) go to their sorted positions.  Each warp takes one contiguous
// run; per-(warp, key) counts and the block's offsets give each warp its base
// per key; inside a warp, lanes with equal keys are ranked by lane (match mask),
// so equal keys keep their input order.
static __global__ void __launch_bounds__(256) k_fused_scatter(const uint64_t* __restrict__ in,
                                                              uint64_t* __restrict__ out,
                                                              const uint32_t* __restrict__ offs,
                                                              const unsigned long long* __restrict__ starts,
                                                              const WsStatus* __restrict__ st, int n_keys) {
    __shared__ uint32_t s_h[8][kFusedKeys];
    const int b = blockIdx.x, nb = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long n_written = st->n_keys;
    const unsigned long long lo = min(starts[b], n_written);
    const unsigned long long hi = (b + 1 < nb) ? min(starts[b + 1], n_written) : n_written;
    const unsigned long long per = (hi - lo + 7) / 8;
    const unsigned long long wlo = min(hi, lo + warp * per), whi = min(hi, wlo + per);
    for (int k = tid; k < n_keys; k += 256)
#pragma unroll
        for (int w = 0; w < 8; ++w) s_h[w][k] = 0;
    __syncthreads();
    for (unsigned long long i = wlo + lane; i < whi; i += 32) atomicAdd(&s_h[warp][(uint32_t)(in[i] >> 32)], 1u);
    __syncthreads();
    for (int k = tid; k < n_keys; k += 256) {
        uint32_t run = offs[(size_t)k * nb + b];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_h[w][k];
            s_h[w][k] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (unsigned long long base = wlo; base < whi; base += 32) {
        const unsigned long long i = base + lane;
        const bool valid = i < whi;
        const uint64_t x = valid ? in[i] : 0ull;
        const uint32_t k = valid ? (uint32_t)(x >> 32) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, k);
        const uint32_t rank = __popc(peers & lt);
        const uint32_t pos = valid ? s_h[warp][k] + rank : 0u;
        __syncwarp();
        if (valid && rank == 0) s_h[warp][k] += __popc(peers);
        __syncwarp();
        if (valid) out[pos] = x;
    }
}

// Whether a key space takes the fused path, and where the sorted lists end up.
inline bool fused_lists(long long n_slots) { return n_slots <= kFusedKeys; }
inline int list_sort_passes(long long n_slots) {
    return fused_lists(n_slots) ? 1 : (bits_for(n_slots) + kRadixBits - 1) / kRadixBits;
}

// Emit, sort and range the lists of n_slots keys; returns the buffer (a or b)
// holding the sorted entries and adds the kernel launches to *launches.  The
// status block must have been cleared by the caller.  key_done (one chunk
// arrival counter per key) must lie between the ranges and the item status
// block, so that the general path's clear of that span zeroes it; the fused path
// zeroes it and gives every empty key one work item, the general path gives
// empty keys none (their outputs must be cleared by the caller).
template <class Op>
uint64_t* build_lists(const Op& op, long long n_rec, long long n_slots, unsigned long long* partials, WsStatus* st,
                      uint64_t* a, uint64_t* b, uint32_t* scratch, long long cap, uint2* ranges, uint32_t* key_done,
                      WsStatus* item_st, uint32_t* item_off, uint64_t* items, long long items_cap, int chunk,
                      ListProf prof, cudaStream_t s, int* launches) {
    const unsigned long long ucap = (unsigned long long)cap;
    if (fused_lists(n_slots)) {
        uint32_t* hist = scratch;
        uint32_t* totals = scratch + (size_t)kRadix * kSortBlocksMax;
        const int nk = (int)n_slots;
        prof_begin(prof.emit, s);
        k_count_chunks<Op><<<kFusedBlocks, 256, 0, s>>>(op, n_rec, partials, st, ucap, totals, nk);
        k_emit_chunks<Op, true><<<kFusedBlocks, 256, 0, s>>>(op, n_rec, partials, a, ucap, hist, totals, nk);
        prof_end(prof.emit, s);
        prof_begin(prof.sort, s);
        k_fused_offsets<<<(nk + 7) / 8, 256, 0, s>>>(hist, totals, kFusedBlocks, nk, (uint32_t)chunk, ranges,
                                                      key_done, item_off, items, (unsigned long long)items_cap,
                                                      item_st);
        k_fused_scatter<<<kFusedBlocks, 256, 0, s>>>(a, b, hist, partials, st, nk);
        prof_end(prof.sort, s);
        *launches += 4;
        return b;
    }
    prof_begin(prof.emit, s);
    k_count_chunks<Op><<<kScanBlocks, 256, 0, s>>>(op, n_rec, partials, st, ucap, nullptr, 0);
    k_emit_chunks<Op, false><<<kScanBlocks, 256, 0, s>>>(op, n_rec, partials, a, ucap, nullptr, nullptr, 0);
    prof_end(prof.emit, s);
    prof_begin(prof.sort, s);
    uint64_t* sorted = radix_sort_u64(a, b, scratch, st, bits_for(n_slots), sort_blocks_for(cap), s);
    prof_end(prof.sort, s);
    prof_begin(prof.ranges, s);
    build_ranges_items(sorted, st, ranges, n_slots, item_st, item_off, items, items_cap, chunk, s);
    prof_end(prof.ranges, s);
    *launches += 2 + 3 * list_sort_passes(n_slots) + 1;
    return sorted;
}

}  // namespace r2g
