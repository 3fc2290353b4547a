// emit.cuh -- count, scan and emit of (key, Gaussian id) list entries, shared by
// the rasterizer (key = tile) and the voxelizer (key = brick), and the list
// builder that turns them into per-key lists sorted by Gaussian id.
//
// Records are processed in list blocks of 256 threads x L records (L grows with
// the record count so that there are at most kMaxListBlocks blocks).  The
// projection kernels run with this blocking: each computes its records' key
// rectangles, counts the entries of its block and calls list_count_tail, whose
// last block to finish turns the block counts into exclusive offsets and writes
// the total and the capacity verdict into the status block.  The emission then
// re-walks each block's records in rounds of 256 and writes every record's
// entries at its offset, in record order (an Op supplies, for record r, its entry
// count, per-record decode data info(r) and key(info, li), the key of its li-th
// entry).  Each round's entries are spread evenly over the block's threads (an
// entry finds its record by binary search over the round's entry offsets), so the
// writes are balanced and contiguous.  Entries beyond the capacity are not written.
//
// Key spaces of at most kFusedKeys keys (one 512^2 view in 16 x 16 tiles, the
// bricks of a TV patch) take a fused path: the emission also counts its block's
// entries per key, and its last block forms each key's base, range and work
// items; one warp per key turns the per-(key, block) counts into scatter
// offsets; a stable scatter (one contiguous run per warp, ranked with warp match
// masks) writes the sorted lists -- three launches after the projection, one pass
// over the entries.  Larger key spaces take the general stable LSD radix sort and
// a range pass.
#pragma once

#include "r2g_internal.cuh"

namespace r2g {

constexpr int kFusedKeys = 1024;
constexpr int kMaxListBlocks = kScanBlocks;  // the block-offset array holds kScanBlocks entries
static_assert((size_t)kFusedKeys * kMaxListBlocks <= (size_t)kRadix * kSortBlocksMax,
              "fused per-(key, block) counts fit the sort scratch");
static_assert(kFusedKeys <= kRadix * 4, "fused key totals fit the sort scratch");

// List blocking of n_rec records: per_thread records per thread, blocks blocks.
struct ListBlocking {
    int per_thread;
    int blocks;
};
inline ListBlocking list_blocking(long long n_rec) {
    const long long per_block = 256ll * kMaxListBlocks;
    const int L = (int)((n_rec + per_block - 1) / per_block);
    const int per = L < 1 ? 1 : L;
    return ListBlocking{per, (int)((n_rec + 256ll * per - 1) / (256ll * per))};
}

// What the projection kernels need to count their blocks' entries.
struct ListCount {
    unsigned long long* partials;  // per-block entry counts -> exclusive offsets (nullptr: no count)
    WsStatus* st;                  // arrival counter, total, verdict (cleared before the launch)
    unsigned long long capacity;
    uint32_t* key_totals;          // fused path: cleared by the last block for the emission
    int n_keys;
};

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

// Called by every thread of a 256-thread projection block with its entry count:
// the block's sum goes to partials[block]; the last block to finish turns all
// gridDim.x sums into exclusive offsets, writes the total and the capacity
// verdict, and clears key_totals.
__device__ __forceinline__ void list_count_tail(const ListCount& lc, unsigned long long mine) {
    __shared__ unsigned long long sm[8];
    __shared__ int s_last;
    const unsigned long long s = block_sum_u64_256(mine, sm);
    if (threadIdx.x == 0) {
        lc.partials[blockIdx.x] = s;
        __threadfence();
        s_last = atomicAdd(&lc.st->blocks_done, 1ull) == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nb = (int)gridDim.x, t = threadIdx.x;
    unsigned long long carry = 0;
    for (int c0 = 0; c0 < nb; c0 += 1024) {  // uniform trip count: the scan syncs the block
        unsigned long long v[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = c0 + 4 * t + q;
            v[q] = i < nb ? __ldcg(lc.partials + i) : 0ull;
            sum += v[q];
        }
        unsigned long long total;
        unsigned long long run = carry + block_excl_scan_u64_256(sum, sm, &total);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = c0 + 4 * t + q;
            if (i < nb) lc.partials[i] = run;
            run += v[q];
        }
        carry += total;
    }
    if (lc.key_totals)
        for (int k = t; k < lc.n_keys; k += 256) lc.key_totals[k] = 0;
    if (t == 0) {
        atomicMax(&lc.st->needed, carry);  // the largest of a call's view chunks
        lc.st->n_keys = carry < lc.capacity ? carry : lc.capacity;
        if (carry > lc.capacity) lc.st->status = R2G_E_CAPACITY;
    }
}

// Where the fused path's last emission block leaves each key's list.
struct FusedKeys {
    uint32_t chunk;           // entries per work item
    uint2* ranges;            // [start, end) per key ([0, 0) when empty)
    uint32_t* key_done;       // chunk arrival counters of the forward, cleared
    uint32_t* item_off;       // first work item of each key
    uint64_t* items;          // (key << 32) | chunk; every empty key gets one item
    unsigned long long items_cap;
    WsStatus* item_st;        // n_keys = item count
    int kd_per_key;           // arrival counters per key (consecutive; 0 taken as 1)
    unsigned long long wait_polls;  // grid-barrier polls before a wait gives up (cooperative builds)
};

// Emission of one block's records (blockIdx.x * per_block .. + per_block), in
// rounds of 256: every record's entries are written at its offset.  HIST (fused
// path): also count the block's written entries per key into hist[key * gridDim.x +
// block] and add them to key_totals.  h: shared [kFusedKeys] (HIST), s_info: shared
// uint4 [256], s_ex: shared [256], sm8: shared [8].
template <class Op, bool HIST>
__device__ __forceinline__ void emit_block(const Op& op, long long n_rec, long long per_block,
                                           unsigned long long running, uint64_t* out,
                                           unsigned long long capacity, uint32_t* __restrict__ hist,
                                           uint32_t* __restrict__ key_totals, int n_keys, uint32_t* h, uint4* s_info,
                                           uint32_t* s_ex, uint32_t* sm8) {
    if (HIST) {
        for (int k = threadIdx.x; k < n_keys; k += 256) h[k] = 0;
        __syncthreads();
    }
    const long long begin = min(n_rec, (long long)blockIdx.x * per_block);
    const long long end = min(n_rec, begin + per_block);
    for (long long base = begin; base < end; base += 256) {
        const long long r = base + threadIdx.x;
        uint32_t c = 0;
        uint4 inf = make_uint4(0u, 0u, 0u, 0u);
        if (r < end) {
            c = op.count(r);
            inf = op.info(r);
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(c, sm8, &tot);
        s_info[threadIdx.x] = inf;
        s_ex[threadIdx.x] = ex;
        __syncthreads();
        // the round's entries, flattened: thread t writes entries t, t + 256, ...
        for (uint32_t e = threadIdx.x; e < tot; e += 256) {
            int lo = 0, hi = 255;  // the record holding entry e: the last k with ex_k <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_ex[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            const uint4 ri = s_info[lo];
            const uint32_t key = op.key(ri, e - s_ex[lo]);
            const unsigned long long off = running + e;
            if (off < capacity) {
                out[off] = ((uint64_t)key << 32) | (uint64_t)ri.w;
                if (HIST) atomicAdd(&h[key], 1u);
            }
        }
        __syncthreads();
        running += tot;
    }
    if (!HIST) return;
    __syncthreads();
    for (int k = threadIdx.x; k < n_keys; k += 256) {
        const uint32_t cnt = h[k];
        hist[(size_t)k * gridDim.x + blockIdx.x] = cnt;
        if (cnt) atomicAdd(&key_totals[k], cnt);
    }
}

// Key bases and item bases (one 256-thread block): exclusive scans over the key
// totals (<= 1024 keys, 4 per thread).  Each key's first entry goes to s_base
// (shared) and/or key_first (global; may be key_totals itself: every thread reads
// its keys' totals before the scans' barriers); with write_items, also every key's
// range, a cleared chunk arrival counter, its first work item and its items, and
// the item count.
__device__ __forceinline__ void key_scan(const uint32_t* key_totals, int n_keys, const FusedKeys& fk,
                                         bool write_items, uint32_t* s_base, uint32_t* key_first, uint32_t* sm8) {
    const int t = threadIdx.x;
    uint32_t tk[4], nc[4], sum = 0, isum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * t + q;
        tk[q] = k < n_keys ? __ldcg(key_totals + k) : 0u;
        nc[q] = k < n_keys ? (tk[q] ? (tk[q] + fk.chunk - 1) / fk.chunk : 1u) : 0u;
        sum += tk[q];
        isum += nc[q];
    }
    uint32_t tot, itot;
    uint32_t base = block_exclusive_scan_256(sum, sm8, &tot);
    uint32_t ibase = block_exclusive_scan_256(isum, sm8, &itot);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * t + q;
        if (k < n_keys) {
            if (s_base) s_base[k] = base;
            if (key_first) key_first[k] = base;
            if (write_items) {
                fk.ranges[k] = tk[q] ? make_uint2(base, base + tk[q]) : make_uint2(0u, 0u);
                const int kd = fk.kd_per_key > 0 ? fk.kd_per_key : 1;
                for (int w = 0; w < kd; ++w) fk.key_done[(size_t)k * kd + w] = 0;
                fk.item_off[k] = ibase;
                for (uint32_t c = 0; c < nc[q]; ++c)
                    if (ibase + c < fk.items_cap) fk.items[ibase + c] = ((uint64_t)(uint32_t)k << 32) | c;
            }
        }
        base += tk[q];
        ibase += nc[q];
    }
    if (write_items && t == 0) fk.item_st->n_keys = itot;
}

// Each block walks its records in rounds of 256 and writes every record's entries
// at its offset (emit_block).  HIST (fused path): the last block to finish (the
// status block's arrival counter, which the count pass left at gridDim.x) turns
// key_totals into each key's first entry (written back into key_totals), range,
// first item and items.
template <class Op, bool HIST>
__global__ void __launch_bounds__(256) k_emit_chunks(Op op, long long n_rec, long long per_block,
                                                     const unsigned long long* partials, uint64_t* out,
                                                     unsigned long long capacity, uint32_t* __restrict__ hist,
                                                     uint32_t* __restrict__ key_totals, int n_keys, WsStatus* st,
                                                     FusedKeys fk) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t h[HIST ? kFusedKeys : 1];
    __shared__ uint4 s_info[256];
    __shared__ uint32_t s_ex[256];
    __shared__ int s_last;
    emit_block<Op, HIST>(op, n_rec, per_block, partials[blockIdx.x], out, capacity, hist, key_totals, n_keys, h,
                         s_info, s_ex, sm);
    if (!HIST) return;
    // the barrier orders every thread's stores before thread 0's release fence
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->blocks_done, 1ull) == 2ull * gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    key_scan(key_totals, n_keys, fk, true, nullptr, key_totals, sm);
}

// The scatter offsets of key k (one warp): offset of (k, emit block b) = the key's
// first entry + entries of key k in earlier blocks (hist row rewritten in place).
constexpr int kMaxRowChunks = (kMaxListBlocks + 31) / 32;
__device__ __forceinline__ void key_offsets(uint32_t* __restrict__ hist, uint32_t key_first, int nb, int k,
                                            int lane) {
    uint32_t* row = hist + (size_t)k * nb;
    uint32_t v[kMaxRowChunks];
#pragma unroll
    for (int c = 0; c < kMaxRowChunks; ++c) {
        const int idx = c * 32 + lane;
        v[c] = idx < nb ? __ldcg(row + idx) : 0u;
    }
    uint32_t running = key_first;
#pragma unroll
    for (int c = 0; c < kMaxRowChunks; ++c) {
        if (c * 32 >= nb) break;
        uint32_t x = v[c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int idx = c * 32 + lane;
        if (idx < nb) row[idx] = running + x - v[c];
        running += __shfl_sync(0xffffffffu, x, 31);
    }
}

// Key bases in shared memory (one 256-thread block, <= 1024 keys, 4 per thread):
// s_base[k] = first entry of key k, s_ibase[k] = its first work item (every key
// gets ceil(entries / chunk) items, an empty key one); [n_keys] hold the totals.
__device__ __forceinline__ void key_bases(const uint32_t* key_totals, int n_keys, uint32_t chunk, uint32_t* s_base,
                                          uint32_t* s_ibase, uint32_t* sm8) {
    const int t = threadIdx.x;
    uint32_t tk[4], nc[4], sum = 0, isum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * t + q;
        tk[q] = k < n_keys ? __ldcg(key_totals + k) : 0u;
        nc[q] = k < n_keys ? (tk[q] ? (tk[q] + chunk - 1) / chunk : 1u) : 0u;
        sum += tk[q];
        isum += nc[q];
    }
    uint32_t tot, itot;
    uint32_t base = block_exclusive_scan_256(sum, sm8, &tot);
    uint32_t ibase = block_exclusive_scan_256(isum, sm8, &itot);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 4 * t + q;
        if (k < n_keys) {
            s_base[k] = base;
            s_ibase[k] = ibase;
        }
        base += tk[q];
        ibase += nc[q];
    }
    if (t == 0) {
        s_base[n_keys] = tot;
        s_ibase[n_keys] = itot;
    }
}

// What the forward and backward read of key k (one warp): its range, cleared chunk
// arrival counters, its first work item and its items (lanes in parallel).
__device__ __forceinline__ void key_publish(const FusedKeys& fk, int k, const uint32_t* s_base,
                                            const uint32_t* s_ibase, int lane) {
    const uint32_t base = s_base[k], tk = s_base[k + 1] - base;
    const uint32_t ibase = s_ibase[k], nc = s_ibase[k + 1] - ibase;
    if (lane == 0) {
        fk.ranges[k] = tk ? make_uint2(base, base + tk) : make_uint2(0u, 0u);
        fk.item_off[k] = ibase;
    }
    const int kd = fk.kd_per_key > 0 ? fk.kd_per_key : 1;
    for (int w = lane; w < kd; w += 32) fk.key_done[(size_t)k * kd + w] = 0;
    for (uint32_t c = lane; c < nc; c += 32)
        if (ibase + c < fk.items_cap) fk.items[ibase + c] = ((uint64_t)(uint32_t)k << 32) | c;
}

// One warp per key k (see key_offsets).
static __global__ void __launch_bounds__(256) k_fused_offsets(uint32_t* __restrict__ hist,
                                                              const uint32_t* __restrict__ key_first, int nb,
                                                              int n_keys) {
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= n_keys) return;
    key_offsets(hist, key_first[k], nb, k, threadIdx.x & 31);
}

// Block b's entries [start_b, start_{b+1}) (clipped to the written count) go to their
// sorted positions.  Each warp takes one contiguous run; per-(warp, key) counts and
// the block's offsets give each warp its base per key; inside a warp, lanes with
// equal keys are ranked by lane (match mask), so equal keys keep their input order.
// s_h: shared [8][kFusedKeys].
template <class Op>
__device__ __forceinline__ void scatter_block(const Op& op, const uint64_t* __restrict__ in,
                                              uint64_t* __restrict__ out, const uint32_t* __restrict__ offs,
                                              unsigned long long lo, unsigned long long hi, int n_keys,
                                              uint32_t (*s_h)[kFusedKeys]) {
    const int b = blockIdx.x, nb = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long per = (hi - lo + 7) / 8;
    const unsigned long long wlo = min(hi, lo + warp * per), whi = min(hi, wlo + per);
    for (int k = tid; k < n_keys; k += 256)
#pragma unroll
        for (int w = 0; w < 8; ++w) s_h[w][k] = 0;
    __syncthreads();
    constexpr int R = 8;  // entries per lane loaded at once
    for (unsigned long long b0 = wlo; b0 < whi; b0 += 32 * R) {
        uint32_t k[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const unsigned long long i = b0 + q * 32 + lane;
            k[q] = i < whi ? (uint32_t)(in[i] >> 32) : 0xffffffffu;
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (k[q] != 0xffffffffu) atomicAdd(&s_h[warp][k[q]], 1u);
    }
    __syncthreads();
    for (int k = tid; k < n_keys; k += 256) {
        uint32_t run = __ldcg(offs + (size_t)k * nb + b);
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_h[w][k];
            s_h[w][k] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (unsigned long long b0 = wlo; b0 < whi; b0 += 32 * R) {
        uint64_t x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const unsigned long long i = b0 + q * 32 + lane;
            x[q] = i < whi ? in[i] : ~0ull;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const bool valid = b0 + q * 32 + lane < whi;
            const uint32_t k = valid ? (uint32_t)(x[q] >> 32) : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, k);
            const uint32_t rank = __popc(peers & lt);
            const uint32_t pos = valid ? s_h[warp][k] + rank : 0u;
            __syncwarp();
            if (valid && rank == 0) s_h[warp][k] += __popc(peers);
            __syncwarp();
            if (valid) {
                out[pos] = x[q];
                op.copy_rec(x[q], pos);  // the entry's record next to it (Op's choice)
            }
        }
    }
}

// One block per emit block (see scatter_block).
template <class Op>
__global__ void __launch_bounds__(256) k_fused_scatter(Op op, const uint64_t* __restrict__ in,
                                                       uint64_t* __restrict__ out, const uint32_t* __restrict__ offs,
                                                       const unsigned long long* __restrict__ starts,
                                                       const WsStatus* __restrict__ st, int n_keys) {
    __shared__ uint32_t s_h[8][kFusedKeys];
    const int b = blockIdx.x;
    const unsigned long long n_written = st->n_keys;
    const unsigned long long lo = min(starts[b], n_written);
    const unsigned long long hi = (b + 1 < (int)gridDim.x) ? min(starts[b + 1], n_written) : n_written;
    scatter_block(op, in, out, offs, lo, hi, n_keys, s_h);
}

// Grid barrier of a cooperative launch (all blocks resident): thread 0 of each
// block arrives on the status block's counter and waits, with a bounded spin, until
// `epoch` x gridDim.x blocks have arrived.  Returns true (in every thread of the
// block) when they have; a wait that gives up after `polls` polls sets
// R2G_E_TIMEOUT and returns false, and the caller's block then leaves the kernel:
// it never arrives at a later barrier, so every other block's later wait gives up
// too, and no block acts on phases that did not finish.  The kernels that consume
// the lists skip their work when the status holds R2G_E_TIMEOUT.
__device__ __forceinline__ bool grid_barrier(WsStatus* st, unsigned int epoch, unsigned long long polls) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long target = (unsigned long long)epoch * gridDim.x;
        // release: the block's writes (ordered before this thread by the block
        // barrier) are visible to any block that observes the arrival
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(&st->grid_sync), "l"(1ull) : "memory");
        unsigned long long spins = 0, seen;
        int ok = 1;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(&st->grid_sync) : "memory");
            if (seen >= target) break;
            if (++spins > polls) {
                atomicExch(&st->status, (int32_t)R2G_E_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        s_ok = ok;
        // the acquire load that saw the last arrival orders the block's later reads
        // (through the block barrier) after every block's writes
    }
    __syncthreads();
    return s_ok != 0;
}

// The key phase of the cooperative builds: the blocks that own keys (warp w of
// block b owns keys b * 8 + w + i * 8 * gridDim.x) form the key bases in shared
// memory; each owning warp turns its key's row of per-block counts into scatter
// offsets and publishes the key's range, arrival counters and work items.  Blocks
// without keys skip the scan.  pool: shared [>= 2 * (n_keys + 1)].
__device__ __forceinline__ void keys_phase(uint32_t* __restrict__ hist, const uint32_t* key_totals, int n_keys,
                                           const FusedKeys& fk, uint32_t* pool, uint32_t* sm8) {
    if ((int)blockIdx.x * 8 >= n_keys) return;  // block-uniform
    uint32_t* s_base = pool;
    uint32_t* s_ibase = pool + kFusedKeys + 1;
    key_bases(key_totals, n_keys, fk.chunk, s_base, s_ibase, sm8);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) fk.item_st->n_keys = s_ibase[n_keys];
    const int lane = threadIdx.x & 31;
    for (int k = blockIdx.x * 8 + (threadIdx.x >> 5); k < n_keys; k += gridDim.x * 8) {
        key_offsets(hist, s_base[k], (int)gridDim.x, k, lane);
        key_publish(fk, k, s_base, s_ibase, lane);
    }
}

// The fused list build in one cooperative launch (grid = the emit blocks): emission
// with per-block key counts; barrier; every block scans the key totals into the
// keys' first entries (block 0 also writes ranges and work items) and the grid's
// warps turn the per-key rows of counts into scatter offsets; barrier; each block
// scatters its entries.  Equal to k_emit_chunks<Op, true> + k_fused_offsets +
// k_fused_scatter, without their launches and the emission's last-block tail.
template <class Op>
__global__ void __launch_bounds__(256) k_lists_coop(Op op, long long n_rec, long long per_block,
                                                    const unsigned long long* __restrict__ partials,
                                                    uint64_t* __restrict__ a, uint64_t* __restrict__ b,
                                                    unsigned long long capacity, uint32_t* __restrict__ hist,
                                                    uint32_t* __restrict__ key_totals, int n_keys, WsStatus* st,
                                                    FusedKeys fk) {
    __shared__ __align__(16) uint32_t pool[8 * kFusedKeys];  // reused by the three phases
    __shared__ uint32_t sm8[8];
    emit_block<Op, true>(op, n_rec, per_block, partials[blockIdx.x], a, capacity, hist, key_totals, n_keys, pool,
                         reinterpret_cast<uint4*>(pool + kFusedKeys), pool + 2 * kFusedKeys, sm8);
    if (!grid_barrier(st, 1, fk.wait_polls)) return;
    keys_phase(hist, key_totals, n_keys, fk, pool, sm8);
    if (!grid_barrier(st, 2, fk.wait_polls)) return;
    const unsigned long long n_written = st->n_keys;
    const unsigned long long lo = min(partials[blockIdx.x], n_written);
    const unsigned long long hi =
        (blockIdx.x + 1 < gridDim.x) ? min(partials[blockIdx.x + 1], n_written) : n_written;
    scatter_block(op, a, b, hist, lo, hi, n_keys, reinterpret_cast<uint32_t(*)[kFusedKeys]>(pool));
}

// The projection and the fused list build in one cooperative launch: each block
// projects its records (proj(r): writes record r, returns its entry count; 0 past
// n_rec) and counts their entries; barrier; every block forms its exclusive entry
// offset and the total from the block counts (block 0 writes the total and the
// capacity verdict into the status block), then emits; barrier; key scan and
// offsets; barrier; scatter.  counts: [gridDim.x] block entry counts (written).
template <class Proj, class Op>
__global__ void __launch_bounds__(256) k_plists_coop(Proj proj, Op op, long long n_rec, int per_thread,
                                                     unsigned long long* __restrict__ counts,
                                                     uint64_t* __restrict__ a, uint64_t* __restrict__ b,
                                                     unsigned long long capacity, uint32_t* __restrict__ hist,
                                                     uint32_t* __restrict__ key_totals, int n_keys, WsStatus* st,
                                                     FusedKeys fk) {
    __shared__ __align__(16) uint32_t pool[8 * kFusedKeys];  // reused by the phases
    __shared__ uint32_t sm8[8];
    __shared__ unsigned long long smu[8];
    unsigned long long cnt = 0;
    for (int l = 0; l < per_thread; ++l) cnt += proj(((long long)blockIdx.x * per_thread + l) * 256 + threadIdx.x);
    const unsigned long long mine = block_sum_u64_256(cnt, smu);
    if (threadIdx.x == 0) counts[blockIdx.x] = mine;
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < n_keys; k += 256) key_totals[k] = 0;
    if (!grid_barrier(st, 1, fk.wait_polls)) return;
    unsigned long long before = 0, total = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) {
        const unsigned long long c = __ldcg(counts + i);
        total += c;
        before += i < (int)blockIdx.x ? c : 0ull;
    }
    before = block_sum_u64_256(before, smu);
    total = block_sum_u64_256(total, smu);
    const unsigned long long written = total < capacity ? total : capacity;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicMax(&st->needed, total);  // the largest of a call's view chunks
        st->n_keys = written;
        if (total > capacity) atomicExch(&st->status, (int32_t)R2G_E_CAPACITY);
    }
    const long long per_block = 256ll * per_thread;
    emit_block<Op, true>(op, n_rec, per_block, before, a, capacity, hist, key_totals, n_keys, pool,
                         reinterpret_cast<uint4*>(pool + kFusedKeys), pool + 2 * kFusedKeys, sm8);
    if (!grid_barrier(st, 2, fk.wait_polls)) return;
    keys_phase(hist, key_totals, n_keys, fk, pool, sm8);
    if (!grid_barrier(st, 3, fk.wait_polls)) return;
    pdl_trigger();  // the forward splat may become resident during the scatter
    const unsigned long long lo = before < written ? before : written;
    const unsigned long long hi = before + mine < written ? before + mine : written;
    scatter_block(op, a, b, hist, lo, hi, n_keys, reinterpret_cast<uint32_t(*)[kFusedKeys]>(pool));
}

// Largest co-resident grid of a kernel of 256-thread blocks on this device (0: no
// cooperative launch); computed once per kernel and device.
template <class K>
int coop_resident(K kern) {
    static int resident[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (resident[dev] == 0) {
        int per_sm = 0, sms = 0, coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess) per_sm = 0;
        resident[dev] = coop && per_sm > 0 ? per_sm * sms : -1;
    }
    return resident[dev] > 0 ? resident[dev] : 0;
}

// Launches k_lists_coop if `blocks` blocks can all be resident on this device;
// false (nothing launched) otherwise.
template <class Op>
bool launch_lists_coop(const Op& op, long long n_rec, long long per_block, const unsigned long long* partials,
                       uint64_t* a, uint64_t* b, unsigned long long capacity, uint32_t* hist, uint32_t* key_totals,
                       int n_keys, WsStatus* st, const FusedKeys& fk, int blocks, cudaStream_t s) {
    if (blocks > coop_resident(k_lists_coop<Op>)) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_lists_coop<Op>, op, n_rec, per_block, partials, a, b, capacity, hist,
                              key_totals, n_keys, st, fk) == cudaSuccess;
}

// Whether a key space takes the fused path, and where the sorted lists end up.
inline bool fused_lists(long long n_slots) { return n_slots <= kFusedKeys; }
inline int list_sort_passes(long long n_slots) {
    return fused_lists(n_slots) ? 1 : (bits_for(n_slots) + kRadixBits - 1) / kRadixBits;
}

// Projection + fused list build in one cooperative launch, with as many records per
// thread as it takes for the grid to be co-resident (at most kMaxListBlocks blocks).
// False (nothing launched) if the key space is not fused or the grid cannot be
// resident; the caller then launches the projection and build_lists.
template <class Proj, class Op>
bool launch_plists_coop(const Proj& proj, const Op& op, long long n_rec, long long n_slots,
                        unsigned long long* counts, uint64_t* a, uint64_t* b, long long cap, uint32_t* scratch,
                        WsStatus* st, uint2* ranges, uint32_t* key_done, WsStatus* item_st, uint32_t* item_off,
                        uint64_t* items, long long items_cap, int chunk, cudaStream_t s, int kd_per_key = 1) {
    if (!fused_lists(n_slots)) return false;
    const int res = coop_resident(k_plists_coop<Proj, Op>);
    const int max_blocks = res < kMaxListBlocks ? res : kMaxListBlocks;
    if (max_blocks <= 0) return false;
    const long long per_thread = (n_rec + 256ll * max_blocks - 1) / (256ll * max_blocks);
    const int per = per_thread < 1 ? 1 : (int)per_thread;
    const int blocks = (int)((n_rec + 256ll * per - 1) / (256ll * per));
    if (blocks < 1 || blocks > max_blocks) return false;
    uint32_t* hist = scratch;
    uint32_t* totals = scratch + (size_t)kRadix * kSortBlocksMax;
    const FusedKeys fk{(uint32_t)chunk, ranges,  key_done,  item_off,    items, (unsigned long long)items_cap,
                       item_st,         kd_per_key, wait_polls()};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_plists_coop<Proj, Op>, proj, op, n_rec, per, counts, a, b,
                              (unsigned long long)cap, hist, totals, (int)n_slots, st, fk) == cudaSuccess;
}

// The count the projection kernel of a list build must make (see list_count_tail).
inline ListCount list_count(long long n_slots, unsigned long long* partials, WsStatus* st, long long cap,
                            uint32_t* scratch) {
    return ListCount{partials, st, (unsigned long long)cap,
                     fused_lists(n_slots) ? scratch + (size_t)kRadix * kSortBlocksMax : nullptr, (int)n_slots};
}

// After the projection kernel (launched with list_blocking(n_rec) and
// list_count(...) on a cleared status block): emit, sort and range the lists of
// n_slots keys; returns the buffer (a or b) holding the sorted entries and adds
// the kernel launches to *launches.  key_done (one chunk arrival counter per key)
// must lie between the ranges and the item status block, so that the general
// path's clear of that span zeroes it; the fused path zeroes it and gives every
// empty key one work item, the general path gives empty keys none (their outputs
// must be cleared by the caller).
template <class Op>
uint64_t* build_lists(const Op& op, long long n_rec, long long n_slots, unsigned long long* partials, WsStatus* st,
                      uint64_t* a, uint64_t* b, uint32_t* scratch, long long cap, uint2* ranges, uint32_t* key_done,
                      WsStatus* item_st, uint32_t* item_off, uint64_t* items, long long items_cap, int chunk,
                      ListProf prof, cudaStream_t s, int* launches, bool allow_coop = true, int kd_per_key = 1) {
    const unsigned long long ucap = (unsigned long long)cap;
    const ListBlocking lb = list_blocking(n_rec);
    const long long per_block = 256ll * lb.per_thread;
    if (fused_lists(n_slots)) {
        uint32_t* hist = scratch;
        uint32_t* totals = scratch + (size_t)kRadix * kSortBlocksMax;
        const int nk = (int)n_slots;
        const FusedKeys fk{(uint32_t)chunk, ranges,  key_done,  item_off,    items, (unsigned long long)items_cap,
                           item_st,         kd_per_key, wait_polls()};
        prof_begin(prof.emit, s);
        if (allow_coop &&
            launch_lists_coop(op, n_rec, per_block, partials, a, b, ucap, hist, totals, nk, st, fk, lb.blocks, s)) {
            prof_end(prof.emit, s);
            *launches += 1;
            return b;
        }
        k_emit_chunks<Op, true><<<lb.blocks, 256, 0, s>>>(op, n_rec, per_block, partials, a, ucap, hist, totals, nk,
                                                          st, fk);
        prof_end(prof.emit, s);
        prof_begin(prof.sort, s);
        k_fused_offsets<<<(nk + 7) / 8, 256, 0, s>>>(hist, totals, lb.blocks, nk);
        k_fused_scatter<Op><<<lb.blocks, 256, 0, s>>>(op, a, b, hist, partials, st, nk);
        prof_end(prof.sort, s);
        *launches += 3;
        return b;
    }
    prof_begin(prof.emit, s);
    k_emit_chunks<Op, false><<<lb.blocks, 256, 0, s>>>(op, n_rec, per_block, partials, a, ucap, nullptr, nullptr, 0,
                                                       st, FusedKeys{});
    prof_end(prof.emit, s);
    prof_begin(prof.sort, s);
    uint64_t* sorted = radix_sort_u64(a, b, scratch, st, bits_for(n_slots), sort_blocks_for(cap), s);
    prof_end(prof.sort, s);
    prof_begin(prof.ranges, s);
    build_ranges_items(sorted, st, ranges, n_slots, item_st, item_off, items, items_cap, chunk, s);
    prof_end(prof.ranges, s);
    *launches += 1 + 3 * list_sort_passes(n_slots) + 1;
    return sorted;
}

// ---------------------------------------------------------------- view-segmented lists
//
// A key space of several views (key = view x kpv + key within the view, kpv <=
// kFusedKeys) whose records are numbered view-major (r = v M + i): the emission, in
// record order, leaves the entries grouped by view, so a stable order by key only
// has to order each view's entries by their key within the view.  Each emission
// block covers a contiguous range of records and so at most a few views: it counts
// its entries per key of those views (its local keys, at most kSegLocalMax) into
// its row of `hist`; one CTA scans the key totals into each key's first entry, its
// range, its work items (every key gets at least one, an empty key's item writes
// zeros) and cleared arrival counters; the offset of (key, block) is the key's first
// entry plus the key's entries in the earlier blocks of its view (a handful); a
// stable scatter (one contiguous run per warp, ranked with warp match masks) writes
// the sorted entries -- one pass over them, where a radix sort of the full keys
// takes two or three.

constexpr int kSegLocalMax = 2 * kFusedKeys;  // local keys of one emission block
constexpr int kSegKeysThreads = 1024;

struct SegKeys {
    long long M;          // records per view
    long long per_block;  // records per emission block
    int kpv;              // keys per view
    int lmax;             // row length of hist / offs (>= every block's local keys)
    int n_keys;           // keys in all
};

// First key and number of local keys of emission block b (0 keys past the records).
__host__ __device__ __forceinline__ void seg_block_keys(const SegKeys& sk, long long n_rec, long long b, int& key_lo,
                                                        int& nloc) {
    const long long r0 = b * sk.per_block;
    const long long r1 = (r0 + sk.per_block < n_rec ? r0 + sk.per_block : n_rec) - 1;
    if (r0 > r1) {
        key_lo = 0;
        nloc = 0;
        return;
    }
    const long long v0 = r0 / sk.M, v1 = r1 / sk.M;
    key_lo = (int)(v0 * sk.kpv);
    nloc = (int)((v1 - v0 + 1) * sk.kpv);
}

// Emission of block blockIdx.x (as emit_block) with the block's entries counted per
// local key into hist_row and added to key_totals.
template <class Op>
__global__ void __launch_bounds__(256) k_emit_seg(Op op, long long n_rec, const unsigned long long* partials,
                                                  uint64_t* __restrict__ out, unsigned long long capacity,
                                                  uint32_t* __restrict__ hist, uint32_t* __restrict__ key_totals,
                                                  SegKeys sk) {
    __shared__ uint32_t h[kSegLocalMax];
    __shared__ uint4 s_info[256];
    __shared__ uint32_t s_ex[256];
    __shared__ uint32_t sm8[8];
    int key_lo, nloc;
    seg_block_keys(sk, n_rec, blockIdx.x, key_lo, nloc);
    for (int k = threadIdx.x; k < nloc; k += 256) h[k] = 0;
    __syncthreads();
    const long long begin = min(n_rec, (long long)blockIdx.x * sk.per_block);
    const long long end = min(n_rec, begin + sk.per_block);
    unsigned long long running = partials[blockIdx.x];
    for (long long base = begin; base < end; base += 256) {
        const long long r = base + threadIdx.x;
        uint32_t c = 0;
        uint4 inf = make_uint4(0u, 0u, 0u, 0u);
        if (r < end) {
            c = op.count(r);
            inf = op.info(r);
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(c, sm8, &tot);
        s_info[threadIdx.x] = inf;
        s_ex[threadIdx.x] = ex;
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < tot; e += 256) {
            int lo = 0, hi = 255;  // the record holding entry e: the last k with ex_k <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_ex[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            const uint4 ri = s_info[lo];
            const uint32_t key = op.key(ri, e - s_ex[lo]);
            const unsigned long long off = running + e;
            if (off < capacity) {
                out[off] = ((uint64_t)key << 32) | (uint64_t)ri.w;
                atomicAdd(&h[key - (uint32_t)key_lo], 1u);
            }
        }
        __syncthreads();
        running += tot;
    }
    uint32_t* row = hist + (size_t)blockIdx.x * sk.lmax;
    for (int k = threadIdx.x; k < nloc; k += 256) {
        const uint32_t cnt = h[k];
        row[k] = cnt;
        if (cnt) atomicAdd(&key_totals[key_lo + k], cnt);
    }
}

// Block-wide exclusive scan of one uint32 per thread for a 1024-thread block.
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t* s32, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s32[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s32[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    *total = s32[31];
    const uint32_t before = (warp > 0 ? s32[warp - 1] : 0u) + x - v;
    __syncthreads();
    return before;
}

// One CTA per view (kpv <= kSegKeysThreads keys, one per thread): the view's key
// totals -> each key's first entry (key_first), range, first work item,
// items, and cleared arrival counters.  The view's first entry and first item are the
// sums over the earlier views' keys, which each CTA forms itself; the last view's CTA
// writes the item count into item_st.
static __global__ void __launch_bounds__(kSegKeysThreads) k_seg_keys(const uint32_t* __restrict__ key_totals,
                                                                     uint32_t* __restrict__ key_first, int kpv,
                                                                     FusedKeys fk) {
    __shared__ uint32_t s32[32];
    const int v = blockIdx.x, t = threadIdx.x;
    const uint32_t chunk = fk.chunk;
    uint32_t before = 0, ibefore = 0;  // this thread's share of the earlier views' entries and items
    for (int u = 0; u < v; ++u)
        if (t < kpv) {
            const uint32_t x = __ldcg(key_totals + (size_t)u * kpv + t);
            before += x;
            ibefore += x ? (x + chunk - 1) / chunk : 1u;
        }
    uint32_t vb, vib;
    block_excl_scan_1024(before, s32, &vb);
    block_excl_scan_1024(ibefore, s32, &vib);
    const int k = v * kpv + t;
    const uint32_t tk = t < kpv ? __ldcg(key_totals + k) : 0u;
    const uint32_t nc = t < kpv ? (tk ? (tk + chunk - 1) / chunk : 1u) : 0u;
    uint32_t vt, vit;
    const uint32_t base = vb + block_excl_scan_1024(tk, s32, &vt);
    const uint32_t ibase = vib + block_excl_scan_1024(nc, s32, &vit);
    if (t < kpv) {
        key_first[k] = base;
        fk.ranges[k] = tk ? make_uint2(base, base + tk) : make_uint2(0u, 0u);
        fk.item_off[k] = ibase;
        const int kd = fk.kd_per_key > 0 ? fk.kd_per_key : 1;
        for (int w = 0; w < kd; ++w) fk.key_done[(size_t)k * kd + w] = 0;
        for (uint32_t c = 0; c < nc; ++c)
            if (ibase + c < fk.items_cap) fk.items[ibase + c] = ((uint64_t)(uint32_t)k << 32) | c;
    }
    if (v == (int)gridDim.x - 1 && t == 0) fk.item_st->n_keys = vib + vit;
}

// offs[b][j] = first entry of block b's local key j: the key's first entry plus its
// entries in the earlier blocks of its view.
static __global__ void __launch_bounds__(256) k_seg_offsets(const uint32_t* __restrict__ hist,
                                                     const uint32_t* __restrict__ key_first,
                                                     uint32_t* __restrict__ offs, long long n_rec, int nb,
                                                     SegKeys sk) {
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    const long long b = t / sk.lmax;
    const int j = (int)(t - b * sk.lmax);
    if (b >= nb) return;
    int key_lo, nloc;
    seg_block_keys(sk, n_rec, b, key_lo, nloc);
    if (j >= nloc) return;
    const int k = key_lo + j;
    const long long v = k / sk.kpv;
    uint32_t run = key_first[k];
    for (long long bb = (v * sk.M) / sk.per_block; bb < b; ++bb) {
        int lo2, n2;
        seg_block_keys(sk, n_rec, bb, lo2, n2);
        run += hist[(size_t)bb * sk.lmax + (k - lo2)];
    }
    offs[(size_t)b * sk.lmax + j] = run;
}

// Block b's entries [start_b, start_{b+1}) (clipped to the written count) to their
// sorted positions: as scatter_block, with the block's local keys.  Dynamic shared
// memory: 8 x lmax words.
template <class Op>
__global__ void __launch_bounds__(256) k_seg_scatter(Op op, const uint64_t* __restrict__ in,
                                                     uint64_t* __restrict__ out, const uint32_t* __restrict__ offs,
                                                     const unsigned long long* __restrict__ starts,
                                                     const WsStatus* __restrict__ st, long long n_rec, SegKeys sk) {
    extern __shared__ uint32_t s_dyn[];
    const int b = blockIdx.x, nb = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int key_lo, nloc;
    seg_block_keys(sk, n_rec, b, key_lo, nloc);
    uint32_t* s_h = s_dyn;  // [8][lmax]
    const unsigned long long n_written = st->n_keys;
    const unsigned long long lo = min(starts[b], n_written);
    const unsigned long long hi = (b + 1 < nb) ? min(starts[b + 1], n_written) : n_written;
    const unsigned long long per = (hi - lo + 7) / 8;
    const unsigned long long wlo = min(hi, lo + warp * per), whi = min(hi, wlo + per);
    for (int k = tid; k < nloc; k += 256)
#pragma unroll
        for (int w = 0; w < 8; ++w) s_h[w * sk.lmax + k] = 0;
    __syncthreads();
    constexpr int R = 8;  // entries per lane loaded at once
    for (unsigned long long b0 = wlo; b0 < whi; b0 += 32 * R) {
        uint32_t k[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const unsigned long long i = b0 + q * 32 + lane;
            k[q] = i < whi ? (uint32_t)(in[i] >> 32) - (uint32_t)key_lo : 0xffffffffu;
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (k[q] != 0xffffffffu) atomicAdd(&s_h[warp * sk.lmax + k[q]], 1u);
    }
    __syncthreads();
    const uint32_t* orow = offs + (size_t)b * sk.lmax;
    for (int k = tid; k < nloc; k += 256) {
        uint32_t run = __ldg(orow + k);
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_h[w * sk.lmax + k];
            s_h[w * sk.lmax + k] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (unsigned long long b0 = wlo; b0 < whi; b0 += 32 * R) {
        uint64_t x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const unsigned long long i = b0 + q * 32 + lane;
            x[q] = i < whi ? in[i] : ~0ull;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const bool valid = b0 + q * 32 + lane < whi;
            const uint32_t k = valid ? (uint32_t)(x[q] >> 32) - (uint32_t)key_lo : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, k);
            const uint32_t rank = __popc(peers & lt);
            const uint32_t pos = valid ? s_h[warp * sk.lmax + k] + rank : 0u;
            __syncwarp();
            if (valid && rank == 0) s_h[warp * sk.lmax + k] += __popc(peers);
            __syncwarp();
            if (valid) {
                out[pos] = x[q];
                op.copy_rec(x[q], pos);  // the entry's record next to it (Op's choice)
            }
        }
    }
}

// The segmented layout of n_rec records, M per view, kpv keys per view, for the
// emission blocking of list_blocking(n_rec); lmax = 0 when it does not apply (the key
// space is fused, or a block could span more than kSegLocalMax local keys).
inline SegKeys seg_keys(long long n_slots, long long M, long long n_rec, int kpv) {
    SegKeys sk{M, 0, kpv, 0, (int)n_slots};
    if (fused_lists(n_slots) || kpv < 1 || kpv > kFusedKeys || M < 1 || n_rec % M != 0 ||
        n_slots != (n_rec / M) * kpv)
        return sk;
    const ListBlocking lb = list_blocking(n_rec);
    sk.per_block = 256ll * lb.per_thread;
    long long span = (sk.per_block + M - 1) / M + 1;  // views one block can meet
    if (span > n_rec / M) span = n_rec / M;
    if (span * kpv > kSegLocalMax) return sk;
    sk.lmax = (int)(span * kpv);
    return sk;
}
inline bool seg_lists(const SegKeys& sk) { return sk.lmax > 0; }

// Scratch words of the segmented build: hist and offs rows for every emission block,
// the key totals and the keys' first entries.
inline size_t seg_scratch_words(const SegKeys& sk) {
    return seg_lists(sk) ? 2 * (size_t)kMaxListBlocks * sk.lmax + 2 * (size_t)sk.n_keys : 0;
}
inline uint32_t* seg_key_totals(uint32_t* seg_scratch, const SegKeys& sk) {
    return seg_scratch + 2 * (size_t)kMaxListBlocks * sk.lmax;
}

// The count the projection kernel of a segmented build must make (it also clears the
// key totals).
inline ListCount seg_list_count(const SegKeys& sk, unsigned long long* partials, WsStatus* st, long long cap,
                                uint32_t* seg_scratch) {
    return ListCount{partials, st, (unsigned long long)cap, seg_key_totals(seg_scratch, sk), sk.n_keys};
}

// After the projection kernel (launched with list_blocking(n_rec) and seg_list_count):
// emission with per-block local counts, key scan, offsets and stable scatter from a
// into b (returned); every key gets a range, cleared arrival counters and at least one
// work item.  Adds the launches to *launches.
template <class Op>
uint64_t* build_lists_seg(const Op& op, long long n_rec, const SegKeys& sk, const unsigned long long* partials,
                          WsStatus* st, uint64_t* a, uint64_t* b, long long cap, uint32_t* seg_scratch, uint2* ranges,
                          uint32_t* key_done, WsStatus* item_st, uint32_t* item_off, uint64_t* items,
                          long long items_cap, int chunk, int kd_per_key, ListProf prof, cudaStream_t s,
                          int* launches) {
    const ListBlocking lb = list_blocking(n_rec);
    uint32_t* hist = seg_scratch;
    uint32_t* offs = seg_scratch + (size_t)kMaxListBlocks * sk.lmax;
    uint32_t* totals = seg_key_totals(seg_scratch, sk);
    prof_begin(prof.emit, s);
    k_emit_seg<Op><<<lb.blocks, 256, 0, s>>>(op, n_rec, partials, a, (unsigned long long)cap, hist, totals, sk);
    prof_end(prof.emit, s);
    prof_begin(prof.sort, s);
    const FusedKeys fk{(uint32_t)chunk, ranges,     key_done,    item_off, items, (unsigned long long)items_cap,
                       item_st,         kd_per_key, wait_polls()};
    uint32_t* first = totals + sk.n_keys;
    k_seg_keys<<<(unsigned)(sk.n_keys / sk.kpv), kSegKeysThreads, 0, s>>>(totals, first, sk.kpv, fk);
    const long long n_off = (long long)lb.blocks * sk.lmax;
    k_seg_offsets<<<(unsigned)((n_off + 255) / 256), 256, 0, s>>>(hist, first, offs, n_rec, lb.blocks, sk);
    const size_t smem = 8 * sizeof(uint32_t) * (size_t)sk.lmax;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaFuncSetAttribute(k_seg_scatter<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(8 * sizeof(uint32_t) * kSegLocalMax));
        attr_set[dev] = true;
    }
    k_seg_scatter<Op><<<lb.blocks, 256, smem, s>>>(op, a, b, offs, partials, st, n_rec, sk);
    prof_end(prof.sort, s);
    *launches += 4;
    return b;
}

}  // namespace r2g
