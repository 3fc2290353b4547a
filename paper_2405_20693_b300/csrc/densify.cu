// densify.cu -- adaptive density control (Sec. 4.2.3): remove empty Gaussians,
// clone or split those whose projected means received large gradients, halving
// the density of both the original and the copy, into a new training state.
//
// Per Gaussian i of the input state (flat layout [quat 4M | mean 3M | scale 3M |
// rho M] for raw, activated, Adam m and Adam v): prune if rho < min_density;
// else densify if the mean of its accumulated |dL/dp^| (normalised device
// coordinates, over the records in which it received a gradient) is at least
// grad_threshold -- clone if its largest scale is at most split_scale, split
// otherwise.  A clone keeps the original (rho / 2) and appends a copy (rho / 2,
// zero Adam moments); a split removes the original and appends two children with
// means p + R(q)(s * z), z standard normal, scales s / split_factor and rho / 2.
// The result holds the survivors in index order, then the copies in the order of
// their originals.  Only the first candidates (index order) that fit in
// max_gaussians are densified; the rest stay as they are.
//
// Split offsets come from a counter-based generator: u_j = ((SplitMix64(seed +
// (j + 1) * 0x9E3779B97F4A7C15) >> 40) + 1/2) / 2^24 (exact in FP32), and child c
// of Gaussian i has z_k = sqrt(-2 ln u_j) cos(2 pi u_{j+1}), j = ((2 i + c) 3 + k) 2
// (Box-Muller).
//
// Kernels (fixed grid of contiguous index ranges, so every pass sees the same
// partition): k_dn_count1 counts the block's non-pruned Gaussians and densify
// candidates; k_dn_scan (one CTA) scans them and fixes the capacity cut;
// k_dn_count2 counts the block's survivors and copies; k_dn_scan again; k_dn_write
// writes the new state at the scanned offsets.
#include <math.h>

#include "adam_math.cuh"
#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr int kDnBlocks = 148 * 6;  // <= 1024: one scan CTA
constexpr unsigned long long kDnGolden = 0x9E3779B97F4A7C15ull;

struct DnState {
    unsigned long long base;     // non-pruned Gaussians
    unsigned long long cand;     // densify candidates
    unsigned long long room;     // candidates that fit
    unsigned long long surv;     // survivors (first part of the output)
    unsigned long long m_new;    // Gaussians in the output
    unsigned long long pad[3];
};

struct DnIn {
    long long M;
    const float *raw, *act, *m, *v, *dgrad, *dcount;
    float grad_threshold, min_density, split_scale, split_factor;
    unsigned long long seed;
    long long cap;
};

// 0 prune, 1 keep, 2 clone, 3 split (before the capacity cut)
__device__ __forceinline__ int dn_kind(const DnIn& a, long long i) {
    const long long M = a.M;
    const float rho = a.act[10 * M + i];
    if (rho < a.min_density) return 0;
    const float n = a.dcount ? a.dcount[i] : 0.f;
    const float g = n > 0.f ? a.dgrad[i] / n : 0.f;
    if (!(g >= a.grad_threshold)) return 1;
    const float* s = a.act + 7 * M + 3 * i;
    return fmaxf(s[0], fmaxf(s[1], s[2])) > a.split_scale ? 3 : 2;
}

__device__ __forceinline__ void dn_range(long long n, long long* lo, long long* hi) {
    const long long per = ((n + gridDim.x - 1) / gridDim.x + 255) / 256 * 256;
    *lo = min(n, (long long)blockIdx.x * per);
    *hi = min(n, *lo + per);
}

__device__ __forceinline__ unsigned int block_sum_256(unsigned int v, unsigned int* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned int t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) k_dn_count1(DnIn a, unsigned int* __restrict__ cnt) {
    __shared__ unsigned int red[8];
    long long lo, hi;
    dn_range(a.M, &lo, &hi);
    unsigned int b = 0, c = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += 256) {
        const int k = dn_kind(a, i);
        b += k > 0;
        c += k >= 2;
    }
    b = block_sum_256(b, red);
    c = block_sum_256(c, red);
    if (threadIdx.x == 0) {
        cnt[blockIdx.x] = b;
        cnt[kDnBlocks + blockIdx.x] = c;
    }
}

// One CTA: exclusive scans of two per-block count arrays (in place); pass 1 fixes
// base, cand and room, pass 2 surv and m_new.
__global__ void __launch_bounds__(1024) k_dn_scan(unsigned int* __restrict__ cnt, int pass, long long cap,
                                                  DnState* __restrict__ st, long long* __restrict__ m_out) {
    __shared__ unsigned int wsum[32];
    __shared__ unsigned long long tot[2];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int arr = 0; arr < 2; ++arr) {
        unsigned int* c = cnt + arr * kDnBlocks;
        const unsigned int v = t < kDnBlocks ? c[t] : 0u;
        unsigned int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const unsigned int s = wsum[lane];
            unsigned int incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            wsum[lane] = incl - s;
            if (lane == 31) tot[arr] = incl;
        }
        __syncthreads();
        if (t < kDnBlocks) c[t] = wsum[warp] + x - v;
        __syncthreads();
    }
    if (t == 0) {
        if (pass == 1) {
            st->base = tot[0];
            st->cand = tot[1];
            st->room = cap > (long long)tot[0] ? (unsigned long long)(cap - (long long)tot[0]) : 0ull;
        } else {
            st->surv = tot[0];
            st->m_new = tot[0] + tot[1];
            *m_out = (long long)(tot[0] + tot[1]);
        }
    }
}

// This thread's Gaussian i (in [lo, hi)): its kind after the capacity cut, from its
// candidate rank (block prefix + in-block rank of the current 256-chunk).
struct DnRank {
    int kind;       // 0 prune, 1 keep, 2 clone, 3 split (after the cut)
    unsigned int surv, kids;  // 1 if it survives; copies it appends
};

__device__ __forceinline__ DnRank dn_cut(int k, unsigned long long cand_rank, unsigned long long room) {
    DnRank r;
    if (k >= 2 && cand_rank >= room) k = 1;
    r.kind = k;
    r.surv = (k == 1 || k == 2) ? 1u : 0u;
    r.kids = k == 2 ? 1u : (k == 3 ? 2u : 0u);
    return r;
}

__global__ void __launch_bounds__(256) k_dn_count2(DnIn a, const unsigned int* __restrict__ cnt1,
                                                   const DnState* __restrict__ st, unsigned int* __restrict__ cnt2) {
    __shared__ uint32_t sm[8];
    __shared__ unsigned int red[8];
    long long lo, hi;
    dn_range(a.M, &lo, &hi);
    unsigned long long cr = cnt1[kDnBlocks + blockIdx.x];  // candidates before this block
    const unsigned long long room = st->room;
    unsigned int s_tot = 0, k_tot = 0;
    for (long long c0 = lo; c0 < hi; c0 += 256) {
        const long long i = c0 + threadIdx.x;
        const int k = i < hi ? dn_kind(a, i) : 0;
        uint32_t nc;
        const uint32_t rank = block_exclusive_scan_256(k >= 2 ? 1u : 0u, sm, &nc);
        const DnRank r = dn_cut(k, cr + rank, room);
        s_tot += r.surv;
        k_tot += r.kids;
        cr += nc;
    }
    s_tot = block_sum_256(s_tot, red);
    k_tot = block_sum_256(k_tot, red);
    if (threadIdx.x == 0) {
        cnt2[blockIdx.x] = s_tot;
        cnt2[kDnBlocks + blockIdx.x] = k_tot;
    }
}

__device__ __forceinline__ float dn_uniform(unsigned long long seed, unsigned long long j) {
    unsigned long long z = seed + (j + 1ull) * kDnGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((float)(unsigned int)(z >> 40) + 0.5f) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ float inv_softplus_f(float y) { return y + logf(-expm1f(-y)); }

struct DnOut {
    float *raw, *act, *m, *v;
};

// Writes Gaussian o of the output (stride Mn) from the given activated values; the
// raw values follow from the activations; Adam moments copied from input index i
// (keep) or zero.
__device__ __forceinline__ void dn_put(const DnIn& a, const DnOut& out, long long Mn, long long o, long long i,
                                       const float q[4], const float p[3], const float s[3], float rho,
                                       bool keep_moments) {
    const long long M = a.M;
    const long long src[11] = {4 * i, 4 * i + 1, 4 * i + 2, 4 * i + 3, 4 * M + 3 * i, 4 * M + 3 * i + 1,
                               4 * M + 3 * i + 2, 7 * M + 3 * i, 7 * M + 3 * i + 1, 7 * M + 3 * i + 2, 10 * M + i};
    const long long dst[11] = {4 * o, 4 * o + 1, 4 * o + 2, 4 * o + 3, 4 * Mn + 3 * o, 4 * Mn + 3 * o + 1,
                               4 * Mn + 3 * o + 2, 7 * Mn + 3 * o, 7 * Mn + 3 * o + 1, 7 * Mn + 3 * o + 2, 10 * Mn + o};
    const float act[11] = {q[0], q[1], q[2], q[3], p[0], p[1], p[2], s[0], s[1], s[2], rho};
#pragma unroll
    for (int e = 0; e < 11; ++e) {
        out.act[dst[e]] = act[e];
        float r = act[e];
        if (e >= 7 && e < 10) r = logf(act[e]);
        if (e == 10) r = inv_softplus_f(act[e]);
        out.raw[dst[e]] = r;
        out.m[dst[e]] = keep_moments ? a.m[src[e]] : 0.f;
        out.v[dst[e]] = keep_moments ? a.v[src[e]] : 0.f;
    }
}

__global__ void __launch_bounds__(256) k_dn_write(DnIn a, const unsigned int* __restrict__ cnt1,
                                                  const unsigned int* __restrict__ cnt2,
                                                  const DnState* __restrict__ st, DnOut out) {
    __shared__ uint32_t sm[8];
    long long lo, hi;
    dn_range(a.M, &lo, &hi);
    const long long M = a.M;
    const long long Mn = (long long)st->m_new;
    const unsigned long long room = st->room, surv_total = st->surv;
    unsigned long long cr = cnt1[kDnBlocks + blockIdx.x];
    unsigned long long so = cnt2[blockIdx.x];                 // survivors before this block
    unsigned long long ko = cnt2[kDnBlocks + blockIdx.x];     // copies before this block
    for (long long c0 = lo; c0 < hi; c0 += 256) {
        const long long i = c0 + threadIdx.x;
        const int k0 = i < hi ? dn_kind(a, i) : 0;
        uint32_t nc, ns, nk;
        const uint32_t rank = block_exclusive_scan_256(k0 >= 2 ? 1u : 0u, sm, &nc);
        const DnRank r = dn_cut(k0, cr + rank, room);
        const uint32_t sof = block_exclusive_scan_256(r.surv, sm, &ns);
        const uint32_t kof = block_exclusive_scan_256(r.kids, sm, &nk);
        if (i < hi && r.kind > 0) {
            float q[4], p[3], s[3];
#pragma unroll
            for (int e = 0; e < 4; ++e) q[e] = a.act[4 * i + e];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                p[e] = a.act[4 * M + 3 * i + e];
                s[e] = a.act[7 * M + 3 * i + e];
            }
            const float rho = a.act[10 * M + i];
            if (r.surv) {
                const long long o = (long long)(so + sof);
                {  // the original: all four arrays as they are (a clone's density halved below)
                    const long long src[11] = {4 * i,     4 * i + 1,     4 * i + 2,     4 * i + 3,
                                               4 * M + 3 * i, 4 * M + 3 * i + 1, 4 * M + 3 * i + 2,
                                               7 * M + 3 * i, 7 * M + 3 * i + 1, 7 * M + 3 * i + 2, 10 * M + i};
                    const long long dst[11] = {4 * o,      4 * o + 1,      4 * o + 2,      4 * o + 3,
                                               4 * Mn + 3 * o, 4 * Mn + 3 * o + 1, 4 * Mn + 3 * o + 2,
                                               7 * Mn + 3 * o, 7 * Mn + 3 * o + 1, 7 * Mn + 3 * o + 2, 10 * Mn + o};
#pragma unroll
                    for (int e = 0; e < 11; ++e) {
                        out.raw[dst[e]] = a.raw[src[e]];
                        out.act[dst[e]] = a.act[src[e]];
                        out.m[dst[e]] = a.m[src[e]];
                        out.v[dst[e]] = a.v[src[e]];
                    }
                    if (r.kind == 2) {
                        out.act[10 * Mn + o] = 0.5f * rho;
                        out.raw[10 * Mn + o] = inv_softplus_f(0.5f * rho);
                    }
                }
            }
            const long long o2 = (long long)(surv_total + ko + kof);
            if (r.kind == 2) {
                dn_put(a, out, Mn, o2, i, q, p, s, 0.5f * rho, false);
            } else if (r.kind == 3) {
                // rotation of the normalised quaternion (w, x, y, z)
                const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
                const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
                const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                                       {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                                       {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
                float sc[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) sc[e] = s[e] / a.split_factor;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float d[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const unsigned long long j = ((unsigned long long)(2 * i + c) * 3ull + (unsigned long long)e) * 2ull;
                        const float u1 = dn_uniform(a.seed, j), u2 = dn_uniform(a.seed, j + 1);
                        d[e] = s[e] * sqrtf(-2.f * logf(u1)) * cosf(6.283185307179586f * u2);
                    }
                    float pc[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) pc[e] = p[e] + R[e][0] * d[0] + R[e][1] * d[1] + R[e][2] * d[2];
                    dn_put(a, out, Mn, o2 + c, i, q, pc, sc, 0.5f * rho, false);
                }
            }
        }
        cr += nc;
        so += ns;
        ko += nk;
    }
}

struct DnLayout {
    size_t state, cnt1, cnt2, total;
};

DnLayout dn_layout() {
    Layout L;
    DnLayout d;
    d.state = L.take(sizeof(DnState));
    d.cnt1 = L.take(sizeof(unsigned int) * 2 * kDnBlocks);
    d.cnt2 = L.take(sizeof(unsigned int) * 2 * kDnBlocks);
    d.total = L.off;
    return d;
}

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API size_t r2g_densify_workspace_size(void) { return dn_layout().total; }

R2G_API r2g_status r2g_densify(int64_t M, const float* raw, const float* act, const float* m, const float* v,
                               const float* dens_grad, const float* dens_count, const r2g_densify_opts* opts,
                               int64_t max_gaussians, float* raw_out, float* act_out, float* m_out, float* v_out,
                               int64_t* m_new, void* ws, size_t ws_bytes, r2g_stream stream) {
    if (M < 1 || M >= (1ll << 31)) return fail(R2G_E_INVAL, "M must be 1 .. 2^31 - 1");
    if (max_gaussians < M || max_gaussians >= (1ll << 31)) return fail(R2G_E_INVAL, "max_gaussians must be M .. 2^31 - 1");
    if (!opts) return fail(R2G_E_INVAL, "opts is NULL");
    if (!(opts->split_factor > 0.f)) return fail(R2G_E_INVAL, "split_factor must be > 0");
    if (!raw || !act || !m || !v || !dens_grad || !dens_count || !raw_out || !act_out || !m_out || !v_out ||
        !m_new || !ws)
        return fail(R2G_E_INVAL, "NULL device pointer");
    const DnLayout L = dn_layout();
    if (ws_bytes < L.total) return fail(R2G_E_INVAL, "densify workspace needs %zu bytes", L.total);
    char* base = static_cast<char*>(ws);
    DnState* st = reinterpret_cast<DnState*>(base + L.state);
    unsigned int* c1 = reinterpret_cast<unsigned int*>(base + L.cnt1);
    unsigned int* c2 = reinterpret_cast<unsigned int*>(base + L.cnt2);
    DnIn a{M, raw, act, m, v, dens_grad, dens_count, opts->grad_threshold, opts->min_density, opts->split_scale,
           opts->split_factor, (unsigned long long)opts->seed, max_gaussians};
    long long* mo = reinterpret_cast<long long*>(m_new);
    prof_begin(P_DENSIFY, stream);
    k_dn_count1<<<kDnBlocks, 256, 0, stream>>>(a, c1);
    k_dn_scan<<<1, 1024, 0, stream>>>(c1, 1, max_gaussians, st, mo);
    k_dn_count2<<<kDnBlocks, 256, 0, stream>>>(a, c1, st, c2);
    k_dn_scan<<<1, 1024, 0, stream>>>(c2, 2, max_gaussians, st, mo);
    k_dn_write<<<kDnBlocks, 256, 0, stream>>>(a, c1, c2, st, DnOut{raw_out, act_out, m_out, v_out});
    prof_end(P_DENSIFY, stream);
    note_launches(5);
    return check_launch("r2g_densify");
}
