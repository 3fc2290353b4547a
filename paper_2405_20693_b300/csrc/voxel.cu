// voxel.cu -- the differentiable voxelizer of R^2-Gaussian on sm_103a (Eq. 4,
// Sec. 4.2.2): sigma(x) = sum_i G_i(x) at the voxel centres of one or more grids,
// through 8^3 bricks, and its adjoint.
//
//   k_vox_project  one thread per (grid, Gaussian) record: the stated FP32 brick
//                  bound and a 64-byte record {c, rho; A..F; rx, ry, rz} in voxel
//                  units, the quadratic form pre-scaled by -log2(e)/2.
//   emit / sort    (brick, Gaussian id) entries, stable radix sort, brick ranges.
//   k_vox_fwd      one CTA (128 threads) per work item (a brick's list cut into
//                  chunks of 32 records, 128 for grids of 2368+ bricks);
//                  records staged in shared memory; each thread owns a run of
//                  4 voxels along x; a warp (two z-slices) skips records whose
//                  gate misses its slab (z span, then the gate's projections on
//                  the xy, xz and yz planes); in a multi-chunk brick
//                  the last chunk to finish sums the chunk volumes in chunk
//                  order.  An empty brick's work item writes zeros.
//   k_vox_bwd      one CTA per group of 16 consecutive sorted entries; the
//                  group's (record, voxel) pairs split evenly over its 128 lanes;
//                  ten moments per record in registers, three vector atomics.
//   k_vox_chain    one thread per Gaussian, looping over grids: moments ->
//                  d rho, d mean, d Sigma^{-1} -> d scale, d quat.
#include <math.h>

#include <algorithm>

#include "emit.cuh"
#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr int kMaxGrids = 64;
constexpr int kB = 8;  // brick edge

struct GridF {
    float o[3], v[3];
    int dims[3], nb[3];
    long long brick_base, vol_base;
};

struct Grids {
    GridF g[kMaxGrids];
    int G;
    long long n_bricks;
};

struct Params {
    const float* mean;
    const float* scale;
    const float* quat;
    const float* rho;
};

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ void rotation(const float q[4], float R[3][3], float qn[4], float& n) {
    const float n2 = fa(fa(fa(fm(q[0], q[0]), fm(q[1], q[1])), fm(q[2], q[2])), fm(q[3], q[3]));
    n = __fsqrt_rn(n2);
    const float w = __fdiv_rn(q[0], n), x = __fdiv_rn(q[1], n), y = __fdiv_rn(q[2], n), z = __fdiv_rn(q[3], n);
    qn[0] = w;
    qn[1] = x;
    qn[2] = y;
    qn[3] = z;
    const float xx = fm(x, x), yy = fm(y, y), zz = fm(z, z), xy = fm(x, y), xz = fm(x, z), yz = fm(y, z);
    const float wx = fm(w, x), wy = fm(w, y), wz = fm(w, z);
    R[0][0] = fs(1.0f, fm(2.0f, fa(yy, zz)));
    R[0][1] = fm(2.0f, fs(xy, wz));
    R[0][2] = fm(2.0f, fa(xz, wy));
    R[1][0] = fm(2.0f, fa(xy, wz));
    R[1][1] = fs(1.0f, fm(2.0f, fa(xx, zz)));
    R[1][2] = fm(2.0f, fs(yz, wx));
    R[2][0] = fm(2.0f, fs(xz, wy));
    R[2][1] = fm(2.0f, fa(yz, wx));
    R[2][2] = fs(1.0f, fm(2.0f, fa(xx, yy)));
}

__device__ __forceinline__ float ceil_clamped(float x, int n) {
    if (!(x > -1.0f)) return -1.0f;
    if (x > (float)n) return (float)n;
    return ceilf(x);
}
__device__ __forceinline__ float floor_clamped(float x, int n) {
    if (!(x > -1.0f)) return -1.0f;
    if (x > (float)n) return (float)n;
    return floorf(x);
}

__device__ __forceinline__ void load_gaussian(const Params& G, long long i, float p[3], float s[3], float q[4]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = G.mean[3 * i + k];
        s[k] = G.scale[3 * i + k];
    }
    const float4 qq = reinterpret_cast<const float4*>(G.quat)[i];
    q[0] = qq.x;
    q[1] = qq.y;
    q[2] = qq.z;
    q[3] = qq.w;
}

// Sigma^{-1} = R diag(1/s^2) R^T
__device__ __forceinline__ void precision(const float R[3][3], const float s[3], float P[3][3]) {
    const float is2[3] = {1.0f / (s[0] * s[0]), 1.0f / (s[1] * s[1]), 1.0f / (s[2] * s[2])};
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) P[j][k] = R[j][0] * R[k][0] * is2[0] + R[j][1] * R[k][1] * is2[1] + R[j][2] * R[k][2] * is2[2];
}

// ------------------------------------------------------------------ records + brick bound

// origin_dev (optional, device): grid g's origin is origin_dev[3g .. 3g+2].
// One (grid, Gaussian) record: returns its brick count.
__device__ __forceinline__ uint32_t vox_project_one(const Params& G, const Grids& grids,
                                                    const float* __restrict__ origin_dev, float Q3, long long M,
                                                    long long r, float4* __restrict__ rec,
                                                    uint4* __restrict__ rect) {
    const int g = (int)(r / M);
    const long long i = r - (long long)g * M;
    const GridF& gf = grids.g[g];
    float org[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) org[k] = origin_dev ? origin_dev[3 * g + k] : gf.o[k];
    float p[3], s[3], q[4], R[3][3], qn[4], qnorm;
    load_gaussian(G, i, p, s, q);
    rotation(q, R, qn, qnorm);
    float Mm[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) Mm[j][k] = fm(R[j][k], s[k]);
    int lo[3], hi[3];
    float c[3], rr[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float skk = fa(fa(fm(Mm[k][0], Mm[k][0]), fm(Mm[k][1], Mm[k][1])), fm(Mm[k][2], Mm[k][2]));
        const float e = __fsqrt_rn(fm(Q3, skk));
        c[k] = fs(__fdiv_rn(fs(p[k], org[k]), gf.v[k]), 0.5f);
        rr[k] = __fdiv_rn(e, gf.v[k]);
        lo[k] = max(0, (int)ceil_clamped(fs(c[k], rr[k]), gf.dims[k]));
        hi[k] = min(gf.dims[k] - 1, (int)floor_clamped(fa(c[k], rr[k]), gf.dims[k]));
        ok = ok && lo[k] <= hi[k];
    }
    float P[3][3];
    precision(R, s, P);
    const float h = -0.5f * kLog2e;
    const float vx = gf.v[0], vy = gf.v[1], vz = gf.v[2];
    float4* o = rec + 4 * r;
    o[0] = make_float4(c[0], c[1], c[2], G.rho[i]);
    o[1] = make_float4(h * P[0][0] * vx * vx, h * P[1][1] * vy * vy, h * P[2][2] * vz * vz, 2.f * h * P[0][1] * vx * vy);
    o[2] = make_float4(2.f * h * P[0][2] * vx * vz, 2.f * h * P[1][2] * vy * vz, 0.f, 0.f);
    o[3] = make_float4(rr[0], rr[1], rr[2], ok ? 1.f : 0.f);
    uint4 rc;
    if (ok) {
        rc.x = (uint32_t)(lo[0] / kB) | ((uint32_t)(hi[0] / kB) << 16);
        rc.y = (uint32_t)(lo[1] / kB) | ((uint32_t)(hi[1] / kB) << 16);
        rc.z = (uint32_t)(lo[2] / kB) | ((uint32_t)(hi[2] / kB) << 16);
    } else {
        rc.x = rc.y = rc.z = 0xffffu;
    }
    rc.w = 0;
    rect[r] = rc;
    return ok ? (uint32_t)((hi[0] / kB - lo[0] / kB + 1) * (hi[1] / kB - lo[1] / kB + 1) *
                           (hi[2] / kB - lo[2] / kB + 1))
              : 0u;
}

// Each thread projects per_thread records, r = ((block * per_thread) + l) * 256 +
// thread, so that a block covers the records of one list block; every record's
// backward moment slot starts at zero; the blocks' brick entries are counted for
// the list build (list_count_tail).
__global__ void __launch_bounds__(256) k_vox_project(Params G, const __grid_constant__ Grids grids,
                                                     const float* __restrict__ origin_dev, float Q3, long long M,
                                                     int per_thread, float4* __restrict__ rec,
                                                     uint4* __restrict__ rect, float4* __restrict__ mom_clear,
                                                     ListCount lc) {
    unsigned long long cnt = 0;
    const long long n_rec = M * grids.G;
    for (int l = 0; l < per_thread; ++l) {
        const long long r = ((long long)blockIdx.x * per_thread + l) * 256 + threadIdx.x;
        if (r >= n_rec) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) mom_clear[3 * r + k] = make_float4(0.f, 0.f, 0.f, 0.f);
        cnt += vox_project_one(G, grids, origin_dev, Q3, M, r, rec, rect);
    }
    list_count_tail(lc, cnt);
}

// The emit needs per-grid brick numbering; it gets the table by value.
struct BrickEmitOp {
    const uint4* rect;
    long long M;

    __device__ __forceinline__ void copy_rec(uint64_t, unsigned long long) const {}
    long long brick_base[kMaxGrids];
    int nbx[kMaxGrids], nby[kMaxGrids];

    __device__ __forceinline__ uint32_t count(long long r) const {
        const uint4 rc = rect[r];
        const int x0 = rc.x & 0xffff, x1 = rc.x >> 16, y0 = rc.y & 0xffff, y1 = rc.y >> 16;
        const int z0 = rc.z & 0xffff, z1 = rc.z >> 16;
        return (x1 >= x0 && y1 >= y0 && z1 >= z0) ? (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1)) : 0u;
    }
    // Per-record decode data: x0 | w << 16, y0 | h << 16, z0 | grid << 16, Gaussian id.
    __device__ __forceinline__ uint4 info(long long r) const {
        const uint4 rc = rect[r];
        const uint32_t x0 = rc.x & 0xffff, x1 = rc.x >> 16, y0 = rc.y & 0xffff, y1 = rc.y >> 16;
        const int g = (int)(r / M);
        return make_uint4(x0 | ((x1 - x0 + 1) << 16), y0 | ((y1 - y0 + 1) << 16), (rc.z & 0xffff) | ((uint32_t)g << 16),
                          (uint32_t)(r - (long long)g * M));
    }
    // Key of the record's li-th entry (bricks in x-fastest order of its box).
    __device__ __forceinline__ uint32_t key(const uint4& inf, uint32_t li) const {
        const uint32_t w = inf.x >> 16, h = inf.y >> 16, g = inf.z >> 16;
        const uint32_t q = li / w, bx = li - q * w;
        const uint32_t bz = q / h, by = q - bz * h;
        return (uint32_t)(brick_base[g] + ((long long)((inf.z & 0xffff) + bz) * nby[g] + (inf.y & 0xffff) + by) *
                                              nbx[g] + (inf.x & 0xffff) + bx);
    }
};

__device__ __forceinline__ int grid_of_brick(const Grids& grids, long long brick) {
    int g = 0;
    while (g + 1 < grids.G && grids.g[g + 1].brick_base <= brick) ++g;
    return g;
}

// ------------------------------------------------------------------ forward

constexpr int kVoxThreads = 128;

// Whether the 2D concave quadratic t = a x^2 + b x y + c y^2 (centre at the origin)
// reaches Tc somewhere on the rectangle [X0, X1] x [Y0, Y1]: the centre, or the
// vertex of t on each edge that faces the centre (t(l d) = l^2 t(d) puts the
// maximum over the rectangle on an edge whose line separates it from the centre).
// A form that is not clearly negative definite reports true.
__device__ __forceinline__ bool quad2_meets_rect(float a, float b, float c, float X0, float X1, float Y0, float Y1,
                                                 float Tc) {
    const float ac4 = 4.0f * a * c;
    if (!(a < 0.0f && c < 0.0f && ac4 - b * b > 0x1p-10f * ac4)) return true;
    const bool inx = X0 <= 0.0f && X1 >= 0.0f, iny = Y0 <= 0.0f && Y1 >= 0.0f;
    if (inx && iny) return true;
    float best = -INFINITY;
    if (!inx) {
        const float xe = X0 > 0.0f ? X0 : X1;
        const float y = fminf(fmaxf(-b * xe * rcp_fast(2.0f * c), Y0), Y1);
        best = fmaf(fmaf(a, xe, b * y), xe, c * y * y);
    }
    if (!iny) {
        const float ye = Y0 > 0.0f ? Y0 : Y1;
        const float x = fminf(fmaxf(-b * ye * rcp_fast(2.0f * a), X0), X1);
        best = fmaxf(best, fmaf(fmaf(a, x, b * ye), x, c * ye * ye));
    }
    return best >= Tc;
}

// The margin below the gate of the voxel culling test, in units of t.
constexpr float kVoxCullMargin = 0.25f;

// Which of a brick's four two-slice slabs (warp w: slices 2w, 2w + 1) a record's
// gate can reach, as a 4-bit mask: the record's z-span first, then its gate's
// projections onto the xy, xz and yz planes (t maximised over the third coordinate:
// a Schur complement of the form) against the slab's rectangles -- a gate that
// misses one projection misses the slab.  lo/hi: the brick's voxel index ranges.
__device__ __forceinline__ uint32_t slab_mask(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                             float bx0, float by0, float bz0, float Tc) {
    const float A = r1.x, B = r1.y, C = r1.z, D = r1.w, E = r2.x, F = r2.y;
    const float X0 = bx0 - r0.x, X1 = X0 + (float)(kB - 1), Y0 = by0 - r0.y, Y1 = Y0 + (float)(kB - 1);
    uint32_t m = 0;
    const bool xy = quad2_meets_rect(A - E * E * rcp_fast(4.0f * C), D - 2.0f * E * F * rcp_fast(4.0f * C),
                                     B - F * F * rcp_fast(4.0f * C), X0, X1, Y0, Y1, Tc);
    if (!xy) return 0u;
    const float i4B = rcp_fast(4.0f * B), i4A = rcp_fast(4.0f * A);
    const float axz = A - D * D * i4B, bxz = E - 2.0f * D * F * i4B, cxz = C - F * F * i4B;
    const float ayz = B - D * D * i4A, byz = F - 2.0f * D * E * i4A, cyz = C - E * E * i4A;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const float zw0 = bz0 + (float)(2 * w), zw1 = zw0 + 1.0f;
        if (r0.z + r3.z < zw0 || r0.z - r3.z > zw1) continue;
        const float Z0 = zw0 - r0.z, Z1 = zw1 - r0.z;
        if (quad2_meets_rect(axz, bxz, cxz, X0, X1, Z0, Z1, Tc) && quad2_meets_rect(ayz, byz, cyz, Y0, Y1, Z0, Z1, Tc))
            m |= 1u << w;
    }
    return m;
}

template <bool COUNT>
__global__ void __launch_bounds__(kVoxThreads, 10) k_vox_fwd(const float4* __restrict__ rec,
                                                         const uint2* __restrict__ ranges,
                                                         const uint64_t* __restrict__ sorted,
                                                         const uint64_t* __restrict__ items,
                                                         const WsStatus* __restrict__ item_st,
                                                         float* __restrict__ partial,
                                                         const uint32_t* __restrict__ item_off,
                                                         uint32_t* __restrict__ key_done, long long M,
                                                         const __grid_constant__ Grids grids, float Tq,
                                                         uint32_t chunk_len, float* __restrict__ vol, WsStatus* st) {
    __shared__ float4 s_r[kVoxThreads][4];
    __shared__ uint32_t s_m[kVoxThreads];  // slabs each staged record's gate can reach
    __shared__ int s_last;
    const unsigned long long it = blockIdx.x;
    // no work items past the count; none at all after a list build that gave up a wait
    if (it >= item_st->n_keys || st->status == R2G_E_TIMEOUT) return;
    const uint64_t item = items[it];
    const long long brick = (long long)(item >> 32);
    const uint32_t chunk = (uint32_t)item;
    const int g = grid_of_brick(grids, brick);
    const GridF& gf = grids.g[g];
    const long long lb = brick - gf.brick_base;
    const int bx = (int)(lb % gf.nb[0]);
    const int by = (int)((lb / gf.nb[0]) % gf.nb[1]);
    const int bz = (int)(lb / ((long long)gf.nb[0] * gf.nb[1]));
    const int t = threadIdx.x;
    const int x0 = bx * kB + (t & 1) * 4, y = by * kB + ((t >> 1) & 7), z = bz * kB + (t >> 4);
    const int warp = t >> 5;
    const float fx0 = (float)x0, fy = (float)y, fz = (float)z;
    const float4* grec = rec + 4 * (size_t)g * (size_t)M;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    unsigned int cnt = 0;
    const uint2 rg = ranges[brick];
    const uint32_t start = rg.x + chunk * chunk_len;
    const uint32_t end = min(start + chunk_len, rg.y);
    const uint32_t nch = (rg.y - rg.x + chunk_len - 1) / chunk_len;
    for (uint32_t base = start; base < end; base += kVoxThreads) {
        const int n = min((uint32_t)kVoxThreads, end - base);
        __syncthreads();
        if (t < n) {
            const uint32_t gid = (uint32_t)sorted[base + t];
            float4 q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = grec[4 * (size_t)gid + k];
#pragma unroll
            for (int k = 0; k < 4; ++k) s_r[t][k] = q[k];
            s_m[t] = slab_mask(q[0], q[1], q[2], q[3], (float)(bx * kB), (float)(by * kB), (float)(bz * kB),
                               Tq - kVoxCullMargin);
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            if (!((s_m[j] >> warp) & 1u)) continue;  // warp-uniform: the gate misses this warp's slab
            const float4 r0 = s_r[j][0];  // cx, cy, cz, rho
            const float4 r1 = s_r[j][1];  // A, B, C, D
            const float4 r2 = s_r[j][2];  // E, F
            const float dy = fy - r0.y, dz = fz - r0.z;
            const float base_q = fmaf(r1.y * dy, dy, fmaf(r1.z * dz, dz, r2.y * dy * dz));
            const float lin = fmaf(r1.w, dy, r2.x * dz);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float dx = fx0 + (float)k - r0.x;
                const float tq = fmaf(fmaf(r1.x, dx, lin), dx, base_q);
                const float e = ex2_approx(tq);
                acc[k] = (tq >= Tq) ? fmaf(r0.w, e, acc[k]) : acc[k];
                if (COUNT) cnt += (tq >= Tq && x0 + k < gf.dims[0] && y < gf.dims[1] && z < gf.dims[2]);
            }
        }
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((t & 31) == 0 && cnt) atomicAdd(&st->pairs, (unsigned long long)cnt);
    }
    if (nch > 1) {
        // several chunks: store this chunk's volume; the last chunk to finish sums
        // the brick's chunk volumes in chunk order
        float4* p = reinterpret_cast<float4*>(partial + it * (size_t)(kB * kB * kB)) + t;
        *p = make_float4(acc[0], acc[1], acc[2], acc[3]);
        // the barrier orders every thread's stores before thread 0's release fence
        __syncthreads();
        if (t == 0) {
            __threadfence();
            s_last = atomicAdd(&key_done[brick], 1u) == nch - 1;
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        const float4* q = reinterpret_cast<const float4*>(partial + (size_t)item_off[brick] * (kB * kB * kB)) + t;
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        for (uint32_t c = 0; c < nch; ++c) {
            const float4 u = __ldcg(q + (size_t)c * (kB * kB * kB / 4));
            sum.x += u.x;
            sum.y += u.y;
            sum.z += u.z;
            sum.w += u.w;
        }
        acc[0] = sum.x;
        acc[1] = sum.y;
        acc[2] = sum.z;
        acc[3] = sum.w;
    }
    if (y < gf.dims[1] && z < gf.dims[2]) {  // one chunk (or none: zeros), or the sum
        float* row = vol + gf.vol_base + ((long long)z * gf.dims[1] + y) * gf.dims[0];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (x0 + k < gf.dims[0]) row[x0 + k] = acc[k];
    }
}

// ------------------------------------------------------------------ backward

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

constexpr int kVoxGroup = 16;  // sorted list entries per backward CTA

// One CTA per group of kVoxGroup consecutive sorted entries, whatever their
// bricks (a grid-stride loop covers every group).  Each record's voxel box inside
// its brick and the grid is w x h x d; the box sizes of the group's records are
// split into kVoxThreads equal contiguous ranges of (record, voxel) pairs, one per
// lane, so a record is shared by several lanes and every lane does the same
// number of pair evaluations.  A lane keeps its current record's ten moments in
// registers and adds them to the record's slot (three vector atomics) when it
// leaves the record or its range ends.  dL/dV is read through the L1 cache.
__global__ void __launch_bounds__(kVoxThreads) k_vox_bwd(const float4* __restrict__ rec,
                                                         const uint64_t* __restrict__ sorted,
                                                         const WsStatus* __restrict__ st, long long M,
                                                         const __grid_constant__ Grids grids, float Tq,
                                                         const float* __restrict__ dvol, float4* __restrict__ mom) {
    __shared__ float4 s_r1[kVoxGroup], s_r2[kVoxGroup];
    __shared__ float4 s_d[kVoxGroup];         // dx, dy, dz of the box's first voxel
    __shared__ int4 s_box[kVoxGroup];         // w, h, n, row stride of the volume
    __shared__ long long s_goff[kVoxGroup];   // dvol index of the box's first voxel
    __shared__ int s_slice[kVoxGroup];        // slice stride of the volume
    __shared__ uint32_t s_ridx[kVoxGroup];    // record index g M + gid
    __shared__ uint32_t s_excl[kVoxGroup + 1];
    // no entries after a list build that gave up a wait (the lists are not valid)
    const unsigned long long n_keys = st->status == R2G_E_TIMEOUT ? 0ull : st->n_keys;
    const unsigned long long n_groups = (n_keys + kVoxGroup - 1) / kVoxGroup;
    const int j = threadIdx.x;
    for (unsigned long long grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
        __syncthreads();  // the previous group's records are no longer read
        if (j < 32) {
            uint32_t n = 0;
            const unsigned long long e = grp * kVoxGroup + j;
            if (j < kVoxGroup && e < n_keys) {
                const uint64_t ent = sorted[e];
                const long long brick = (long long)(ent >> 32);
                const uint32_t gid = (uint32_t)ent;
                const int g = grid_of_brick(grids, brick);
                const GridF& gf = grids.g[g];
                const long long lb = brick - gf.brick_base;
                const int X0 = (int)(lb % gf.nb[0]) * kB;
                const int Y0 = (int)((lb / gf.nb[0]) % gf.nb[1]) * kB;
                const int Z0 = (int)(lb / ((long long)gf.nb[0] * gf.nb[1])) * kB;
                const size_t r = (size_t)g * (size_t)M + gid;
                const float4 r0 = rec[4 * r], r1 = rec[4 * r + 1], r2 = rec[4 * r + 2], r3 = rec[4 * r + 3];
                const int xa = max(0, (int)ceilf(r0.x - r3.x) - X0);
                const int xb = min(min(kB, gf.dims[0] - X0) - 1, (int)floorf(r0.x + r3.x) - X0);
                const int ya = max(0, (int)ceilf(r0.y - r3.y) - Y0);
                const int yb = min(min(kB, gf.dims[1] - Y0) - 1, (int)floorf(r0.y + r3.y) - Y0);
                const int za = max(0, (int)ceilf(r0.z - r3.z) - Z0);
                const int zb = min(min(kB, gf.dims[2] - Z0) - 1, (int)floorf(r0.z + r3.z) - Z0);
                const int w = xb - xa + 1, h = yb - ya + 1, d = zb - za + 1;
                n = (w > 0 && h > 0 && d > 0) ? (uint32_t)(w * h * d) : 0u;
                const int x = X0 + xa, y = Y0 + ya, z = Z0 + za;
                s_r1[j] = r1;
                s_r2[j] = r2;
                s_d[j] = make_float4((float)x - r0.x, (float)y - r0.y, (float)z - r0.z, 0.f);
                s_box[j] = make_int4(max(w, 1), max(h, 1), (int)n, gf.dims[0]);
                s_slice[j] = gf.dims[0] * gf.dims[1];
                s_goff[j] = n ? gf.vol_base + ((long long)z * gf.dims[1] + y) * gf.dims[0] + x : 0;
                s_ridx[j] = (uint32_t)r;
            } else if (j < kVoxGroup) {
                s_box[j] = make_int4(1, 1, 0, 0);
            }
            const uint32_t incl = warp_incl_scan(n);
            if (j < kVoxGroup) s_excl[j] = incl - n;
            if (j == 31) s_excl[kVoxGroup] = incl;
        }
        __syncthreads();
        const uint32_t T = s_excl[kVoxGroup];
        const uint32_t per = (T + kVoxThreads - 1) / kVoxThreads;
        const uint32_t p0 = j * per, p1 = min(T, p0 + per);
        if (p0 >= p1) continue;
        // the record holding pair p0: the largest k with excl_k <= p0 (it is non-empty)
        int lo = 0, hi = kVoxGroup - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_excl[mid] <= p0) lo = mid;
            else hi = mid - 1;
        }
        int k = lo;
        float4 r1 = s_r1[k], r2 = s_r2[k], d0 = s_d[k];
        int4 box = s_box[k];
        int slice = s_slice[k];
        uint32_t rec_end = s_excl[k] + (uint32_t)box.z;
        const int li = (int)(p0 - s_excl[k]);
        const int zz = li / (box.x * box.y);
        const int rem = li - zz * box.x * box.y;
        const int yy = rem / box.x;
        int xx = rem - yy * box.x;
        int cy = yy;  // rows done inside the current z-slice
        float dx = d0.x + (float)xx, dy = d0.y + (float)yy, dz = d0.z + (float)zz;
        float base_q = fmaf(r1.y * dy, dy, fmaf(r1.z * dz, dz, r2.y * dy * dz));
        float lin = fmaf(r1.w, dy, r2.x * dz);
        const float* grow = dvol + s_goff[k] + (long long)zz * slice + (long long)yy * box.w;
        float S0 = 0.f, Sx = 0.f, Sy = 0.f, Sz = 0.f, Sxx = 0.f, Syy = 0.f, Szz = 0.f, Sxy = 0.f, Sxz = 0.f,
              Syz = 0.f;
        for (uint32_t p = p0; p < p1; ++p) {
            const float tq = fmaf(fmaf(r1.x, dx, lin), dx, base_q);
            const float ev = ex2_approx(tq);
            const float w = (tq >= Tq) ? __ldg(grow + xx) * ev : 0.0f;
            const float wx = w * dx, wy = w * dy, wz = w * dz;
            S0 += w;
            Sx += wx;
            Sy += wy;
            Sz += wz;
            Sxx = fmaf(wx, dx, Sxx);
            Syy = fmaf(wy, dy, Syy);
            Szz = fmaf(wz, dz, Szz);
            Sxy = fmaf(wx, dy, Sxy);
            Sxz = fmaf(wx, dz, Sxz);
            Syz = fmaf(wy, dz, Syz);
            ++xx;
            dx += 1.0f;
            if (xx == box.x) {  // next row (and slice) of the box
                xx = 0;
                dx -= (float)box.x;
                ++cy;
                dy += 1.0f;
                grow += box.w;
                if (cy == box.y) {
                    cy = 0;
                    dy -= (float)box.y;
                    dz += 1.0f;
                    grow += slice - (long long)box.y * box.w;
                }
                base_q = fmaf(r1.y * dy, dy, fmaf(r1.z * dz, dz, r2.y * dy * dz));
                lin = fmaf(r1.w, dy, r2.x * dz);
            }
            if (p + 1 == rec_end && p + 1 < p1) {  // next record
                float4* m = mom + 3 * (size_t)s_ridx[k];
                atomicAdd(&m[0], make_float4(S0, Sx, Sy, Sz));
                atomicAdd(&m[1], make_float4(Sxx, Syy, Szz, Sxy));
                atomicAdd(reinterpret_cast<float2*>(&m[2]), make_float2(Sxz, Syz));
                S0 = Sx = Sy = Sz = Sxx = Syy = Szz = Sxy = Sxz = Syz = 0.f;
                do {
                    ++k;
                } while (s_box[k].z == 0);
                r1 = s_r1[k];
                r2 = s_r2[k];
                d0 = s_d[k];
                box = s_box[k];
                slice = s_slice[k];
                rec_end += (uint32_t)box.z;
                xx = 0;
                cy = 0;
                dx = d0.x;
                dy = d0.y;
                dz = d0.z;
                base_q = fmaf(r1.y * dy, dy, fmaf(r1.z * dz, dz, r2.y * dy * dz));
                lin = fmaf(r1.w, dy, r2.x * dz);
                grow = dvol + s_goff[k];
            }
        }
        float4* m = mom + 3 * (size_t)s_ridx[k];
        atomicAdd(&m[0], make_float4(S0, Sx, Sy, Sz));
        atomicAdd(&m[1], make_float4(Sxx, Syy, Szz, Sxy));
        atomicAdd(reinterpret_cast<float2*>(&m[2]), make_float2(Sxz, Syz));
    }
}

__device__ __forceinline__ void quat_grad(const float qn[4], float qnorm, const float g[3][3], float dq[4]) {
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    float dw = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
    dy -= 4.f * y * g[0][0]; dz -= 4.f * z * g[0][0];
    dx += 2.f * y * g[0][1]; dy += 2.f * x * g[0][1]; dw -= 2.f * z * g[0][1]; dz -= 2.f * w * g[0][1];
    dx += 2.f * z * g[0][2]; dz += 2.f * x * g[0][2]; dw += 2.f * y * g[0][2]; dy += 2.f * w * g[0][2];
    dx += 2.f * y * g[1][0]; dy += 2.f * x * g[1][0]; dw += 2.f * z * g[1][0]; dz += 2.f * w * g[1][0];
    dx -= 4.f * x * g[1][1]; dz -= 4.f * z * g[1][1];
    dy += 2.f * z * g[1][2]; dz += 2.f * y * g[1][2]; dw -= 2.f * x * g[1][2]; dx -= 2.f * w * g[1][2];
    dx += 2.f * z * g[2][0]; dz += 2.f * x * g[2][0]; dw -= 2.f * y * g[2][0]; dy -= 2.f * w * g[2][0];
    dy += 2.f * z * g[2][1]; dz += 2.f * y * g[2][1]; dw += 2.f * x * g[2][1]; dx += 2.f * w * g[2][1];
    dx -= 4.f * x * g[2][2]; dy -= 4.f * y * g[2][2];
    const float dot = w * dw + x * dx + y * dy + z * dz;
    dq[0] = (dw - w * dot) / qnorm;
    dq[1] = (dx - x * dot) / qnorm;
    dq[2] = (dy - y * dot) / qnorm;
    dq[3] = (dz - z * dot) / qnorm;
}

// ASSIGN: write the gradients (zeros where the Gaussian has no moments) instead
// of adding to them.
template <bool ASSIGN>
__global__ void __launch_bounds__(128) k_vox_chain(Params G, const __grid_constant__ Grids grids, long long M,
                                                   float4* __restrict__ mom, float* __restrict__ dmean,
                                                   float* __restrict__ dscale, float* __restrict__ dquat,
                                                   float* __restrict__ drho) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    float p[3], s[3], q[4], R[3][3], qn[4], qnorm;
    load_gaussian(G, i, p, s, q);
    rotation(q, R, qn, qnorm);
    float P[3][3];
    precision(R, s, P);
    const float rho = G.rho[i];
    float gp[3] = {0.f, 0.f, 0.f}, dP[3][3] = {{0.f}}, grho = 0.f;
    bool any = false;
    for (int g = 0; g < grids.G; ++g) {
        const size_t r = (size_t)g * (size_t)M + (size_t)i;
        const float4 m0 = mom[3 * r], m1 = mom[3 * r + 1], m2 = mom[3 * r + 2];
        if (m0.x == 0.f && m0.y == 0.f && m0.z == 0.f && m0.w == 0.f && m1.x == 0.f && m1.y == 0.f && m1.z == 0.f &&
            m1.w == 0.f && m2.x == 0.f && m2.y == 0.f)
            continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) mom[3 * r + k] = make_float4(0.f, 0.f, 0.f, 0.f);  // consumed
        any = true;
        const GridF& gf = grids.g[g];
        const float v[3] = {gf.v[0], gf.v[1], gf.v[2]};
        const float S1[3] = {m0.y, m0.z, m0.w};
        const float S2[3][3] = {{m1.x, m1.w, m2.x}, {m1.w, m1.y, m2.y}, {m2.x, m2.y, m1.z}};
        grho += m0.x;
        // d c = rho P_vox S1, c_k = (p_k - o_k)/v_k - 1/2, P_vox_jk = P_jk v_j v_k
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float dc = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) dc += P[j][k] * v[j] * v[k] * S1[k];
            gp[j] += rho * dc / v[j];
        }
        // d P_jk = -1/2 rho S2_jk v_j v_k
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) dP[j][k] += -0.5f * rho * S2[j][k] * v[j] * v[k];
    }
    if (!any) {
        if (ASSIGN) {
#pragma unroll
            for (int k = 0; k < 3; ++k) dmean[3 * i + k] = dscale[3 * i + k] = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) dquat[4 * i + k] = 0.f;
            drho[i] = 0.f;
        }
        return;
    }
    // P = N N^T, N = R diag(1/s): dN = (dP + dP^T) N
    float gR[3][3], gs[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float dN = 0.f;
#pragma unroll
            for (int m = 0; m < 3; ++m) dN += (dP[j][m] + dP[m][j]) * R[m][k] / s[k];
            gR[j][k] = dN / s[k];
            gs[k] += -dN * R[j][k] / (s[k] * s[k]);
        }
    float gq[4];
    quat_grad(qn, qnorm, gR, gq);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dmean[3 * i + k] = ASSIGN ? gp[k] : dmean[3 * i + k] + gp[k];
        dscale[3 * i + k] = ASSIGN ? gs[k] : dscale[3 * i + k] + gs[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) dquat[4 * i + k] = ASSIGN ? gq[k] : dquat[4 * i + k] + gq[k];
    drho[i] = ASSIGN ? grho : drho[i] + grho;
}

// ------------------------------------------------------------------ host side

struct VoxLayout {
    size_t status, rec, rect, partials, ranges, key_done, mom, scratch, item_status, item_off, fixed;
    long long n_rec, n_bricks, n_vox;
};

r2g_status make_grids(int32_t G, const r2g_grid* grids, Grids& out) {
    if (G < 1 || G > kMaxGrids) return fail(R2G_E_INVAL, "G = %d out of range [1, %d]", G, kMaxGrids);
    if (!grids) return fail(R2G_E_INVAL, "grids must not be NULL");
    out.G = G;
    long long bb = 0, vb = 0;
    for (int g = 0; g < G; ++g) {
        GridF& f = out.g[g];
        for (int k = 0; k < 3; ++k) {
            if (grids[g].dims[k] < 1 || grids[g].dims[k] > 4096)
                return fail(R2G_E_INVAL, "grid %d dims[%d] = %d out of range", g, k, grids[g].dims[k]);
            if (!(grids[g].voxel[k] > 0.f)) return fail(R2G_E_INVAL, "grid %d voxel size must be > 0", g);
            f.o[k] = grids[g].origin[k];
            f.v[k] = grids[g].voxel[k];
            f.dims[k] = grids[g].dims[k];
            f.nb[k] = (f.dims[k] + kB - 1) / kB;
        }
        f.brick_base = bb;
        f.vol_base = vb;
        bb += (long long)f.nb[0] * f.nb[1] * f.nb[2];
        vb += (long long)f.dims[0] * f.dims[1] * f.dims[2];
    }
    if (bb >= (1ll << 31)) return fail(R2G_E_INVAL, "too many bricks");
    out.n_bricks = bb;
    for (int g = G; g < kMaxGrids; ++g) out.g[g] = out.g[G - 1];
    return R2G_OK;
}

VoxLayout vox_layout(int64_t M, const Grids& grids) {
    VoxLayout L;
    L.n_rec = (long long)M * grids.G;
    L.n_bricks = grids.n_bricks;
    const GridF& last = grids.g[grids.G - 1];
    L.n_vox = last.vol_base + (long long)last.dims[0] * last.dims[1] * last.dims[2];
    Layout lay;
    L.status = lay.take(sizeof(WsStatus));
    L.rec = lay.take(64 * (size_t)L.n_rec);
    L.rect = lay.take(16 * (size_t)L.n_rec);
    L.partials = lay.take(8 * (size_t)kScanBlocks);
    L.ranges = lay.take(8 * (size_t)L.n_bricks);
    L.key_done = lay.take(4 * (size_t)L.n_bricks);  // chunk arrival counters of the forward
    L.item_status = lay.take(sizeof(WsStatus));      // ranges .. item status are cleared together
    L.mom = lay.take(48 * (size_t)L.n_rec);
    L.scratch = lay.take(sort_scratch_bytes());
    L.item_off = lay.take(4 * (size_t)L.n_bricks);
    L.fixed = lay.off;
    return L;
}

struct VTail {
    size_t a, b, items, partial, end;
    long long icap;
};

// List entries per brick work item of the forward: kVoxChunk for small grids (TV
// patches: enough items to fill the GPU), kVoxChunkLarge once the bricks alone give
// several waves (a full volume), where longer items mean fewer per-chunk volumes to
// write and sum.
constexpr int kVoxChunkLarge = 128;
inline int vox_chunk(long long n_bricks) { return n_bricks >= 148 * 16 ? kVoxChunkLarge : kVoxChunk; }

VTail vox_tail(const VoxLayout& L, long long cap) {
    VTail t;
    t.icap = items_capacity(L.n_bricks, cap, vox_chunk(L.n_bricks));
    Layout lay;
    lay.off = L.fixed;
    t.a = lay.take(8 * (size_t)cap);
    t.b = lay.take(8 * (size_t)cap);
    t.items = lay.take(8 * (size_t)t.icap);
    t.partial = lay.take(4 * (size_t)(kB * kB * kB) * (size_t)t.icap);
    t.end = lay.off;
    return t;
}

long long vox_capacity(const VoxLayout& L, size_t ws_bytes) {
    if (ws_bytes <= L.fixed) return 0;
    const double per = 16.0 + (8.0 + 4.0 * kB * kB * kB) / vox_chunk(L.n_bricks);
    const double fixed_tail = (double)L.n_bricks * (8.0 + 4.0 * kB * kB * kB) + 4096.0;
    const double est = ((double)(ws_bytes - L.fixed) - fixed_tail) / per;
    long long cap = est > 0 ? ((long long)est / 32) * 32 : 0;
    if (cap > 0xffffffe0ll) cap = 0xffffffe0ll;
    while (cap + 32 <= 0xffffffe0ll && vox_tail(L, cap + 32).end <= ws_bytes) cap += 32;
    while (cap > 0 && vox_tail(L, cap).end > ws_bytes) cap -= 32;
    return cap;
}

uint64_t* vox_sorted(char* base, const VoxLayout& L, const VTail& t) {
    return reinterpret_cast<uint64_t*>(base + ((list_sort_passes(L.n_bricks) & 1) ? t.b : t.a));
}

r2g_status check_params(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho) {
    if (M < 1 || M >= (int64_t(1) << 31)) return fail(R2G_E_INVAL, "M = %lld out of range", (long long)M);
    if (!mean || !scale || !quat || !rho) return fail(R2G_E_INVAL, "NULL parameter pointer");
    if (reinterpret_cast<uintptr_t>(quat) % 16) return fail(R2G_E_INVAL, "quat must be 16-byte aligned");
    return R2G_OK;
}

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API size_t r2g_voxel_workspace_size(int64_t M, int32_t G, const r2g_grid* grids, int64_t key_capacity) {
    Grids gr;
    if (M < 1 || M >= (int64_t(1) << 31) || make_grids(G, grids, gr) != R2G_OK) return 0;
    if ((long long)M * G >= (1ll << 31)) return 0;
    if (key_capacity < 1 || key_capacity > 0xffffffe0ll) return 0;
    const VoxLayout L = vox_layout(M, gr);
    return vox_tail(L, key_capacity).end;
}

namespace r2g {
r2g_status voxelize_impl(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                         int32_t G, const r2g_grid* grids, const float* origin_dev, float Q3, float* vol, void* ws,
                         size_t ws_bytes, cudaStream_t stream, bool count, bool separate_lists) {
    r2g_status e = check_params(M, mean, scale, quat, rho);
    if (e) return e;
    Grids gr;
    if ((e = make_grids(G, grids, gr))) return e;
    if ((long long)M * G >= (1ll << 31)) return fail(R2G_E_INVAL, "M * G must be < 2^31");
    if (!(Q3 > 0.f)) return fail(R2G_E_INVAL, "Q3 must be > 0");
    if (!vol || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    const VoxLayout L = vox_layout(M, gr);
    const long long cap = vox_capacity(L, ws_bytes);
    if (cap < 32) return fail(R2G_E_INVAL, "workspace of %zu bytes holds no list entries", ws_bytes);
    const VTail T = vox_tail(L, cap);
    char* base = static_cast<char*>(ws);
    WsStatus* st = reinterpret_cast<WsStatus*>(base + L.status);
    float4* rec = reinterpret_cast<float4*>(base + L.rec);
    uint4* rect = reinterpret_cast<uint4*>(base + L.rect);
    auto* partials = reinterpret_cast<unsigned long long*>(base + L.partials);
    uint2* ranges = reinterpret_cast<uint2*>(base + L.ranges);
    uint32_t* scratch = reinterpret_cast<uint32_t*>(base + L.scratch);
    uint64_t* a = reinterpret_cast<uint64_t*>(base + T.a);
    uint64_t* b = reinterpret_cast<uint64_t*>(base + T.b);
    WsStatus* item_st = reinterpret_cast<WsStatus*>(base + L.item_status);
    uint32_t* item_off = reinterpret_cast<uint32_t*>(base + L.item_off);
    uint32_t* key_done = reinterpret_cast<uint32_t*>(base + L.key_done);
    uint64_t* items = reinterpret_cast<uint64_t*>(base + T.items);
    float* partial = reinterpret_cast<float*>(base + T.partial);
    // the status block (with the arrival counters of the list passes) starts cleared
    cudaMemsetAsync(st, 0, sizeof(WsStatus), stream);
    // the general list path gives empty bricks no work item: their voxels stay zero
    if (!fused_lists(L.n_bricks)) cudaMemsetAsync(vol, 0, sizeof(float) * (size_t)L.n_vox, stream);
    Params P{mean, scale, quat, rho};
    prof_begin(P_VOX_PROJECT, stream);
    const ListBlocking lb = list_blocking(L.n_rec);
    k_vox_project<<<(unsigned)lb.blocks, 256, 0, stream>>>(P, gr, origin_dev, Q3, M, lb.per_thread, rec, rect,
                                                            reinterpret_cast<float4*>(base + L.mom),
                                                            list_count(L.n_bricks, partials, st, cap, scratch));
    prof_end(P_VOX_PROJECT, stream);
    BrickEmitOp op;
    op.rect = rect;
    op.M = M;
    for (int g = 0; g < kMaxGrids; ++g) {
        op.brick_base[g] = gr.g[g].brick_base;
        op.nbx[g] = gr.g[g].nb[0];
        op.nby[g] = gr.g[g].nb[1];
    }
    int launches = 0;
    uint64_t* sorted = build_lists(op, L.n_rec, L.n_bricks, partials, st, a, b, scratch, cap, ranges, key_done,
                                   item_st, item_off, items, T.icap, vox_chunk(L.n_bricks),
                                   ListProf{P_VOX_EMIT, P_VOX_SORT, P_VOX_RANGES}, stream, &launches, !separate_lists);
    const float Tq = -0.5f * kLog2e * Q3;
    note_launches(1 + launches + 1);
    prof_begin(P_VOX_FWD, stream);
    if (count)
        k_vox_fwd<true><<<(unsigned)T.icap, kVoxThreads, 0, stream>>>(rec, ranges, sorted, items, item_st, partial,
                                                                       item_off, key_done, M, gr, Tq,
                                                                       (uint32_t)vox_chunk(L.n_bricks), vol, st);
    else
        k_vox_fwd<false><<<(unsigned)T.icap, kVoxThreads, 0, stream>>>(rec, ranges, sorted, items, item_st, partial,
                                                                        item_off, key_done, M, gr, Tq,
                                                                        (uint32_t)vox_chunk(L.n_bricks), vol, st);
    prof_end(P_VOX_FWD, stream);
    return check_launch("r2g_voxelize");
}
}  // namespace r2g

R2G_API r2g_status r2g_voxelize(int64_t M, const float* mean, const float* scale, const float* quat,
                                const float* rho, int32_t G, const r2g_grid* grids, float Q3, float* vol, void* ws,
                                size_t ws_bytes, r2g_stream stream) {
    return voxelize_impl(M, mean, scale, quat, rho, G, grids, nullptr, Q3, vol, ws, ws_bytes, stream, false);
}

R2G_API r2g_status r2g_voxelize_counted(int64_t M, const float* mean, const float* scale, const float* quat,
                                        const float* rho, int32_t G, const r2g_grid* grids, float Q3, float* vol,
                                        void* ws, size_t ws_bytes, r2g_stream stream) {
    return voxelize_impl(M, mean, scale, quat, rho, G, grids, nullptr, Q3, vol, ws, ws_bytes, stream, true);
}


namespace r2g {
r2g_status voxelize_backward_impl(int64_t M, const float* mean, const float* scale, const float* quat,
                                  const float* rho, int32_t G, const r2g_grid* grids, float Q3, const float* dvol,
                                  float* dmean, float* dscale, float* dquat, float* drho, void* ws, size_t ws_bytes,
                                  cudaStream_t stream, int parts) {
    r2g_status e = check_params(M, mean, scale, quat, rho);
    if (e) return e;
    Grids gr;
    if ((e = make_grids(G, grids, gr))) return e;
    if ((long long)M * G >= (1ll << 31)) return fail(R2G_E_INVAL, "M * G must be < 2^31");
    if (!dvol || !dmean || !dscale || !dquat || !drho || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    const VoxLayout L = vox_layout(M, gr);
    const long long cap = vox_capacity(L, ws_bytes);
    if (cap < 32) return fail(R2G_E_INVAL, "workspace of %zu bytes holds no list entries", ws_bytes);
    const VTail T = vox_tail(L, cap);
    char* base = static_cast<char*>(ws);
    const float4* rec = reinterpret_cast<const float4*>(base + L.rec);
    float4* mom = reinterpret_cast<float4*>(base + L.mom);
    const uint64_t* sorted = vox_sorted(base, L, T);
    const WsStatus* st = reinterpret_cast<const WsStatus*>(base + L.status);
    if (parts & kVoxBwdMoments) {
        const float Tq = -0.5f * kLog2e * Q3;
        const long long groups = (cap + kVoxGroup - 1) / kVoxGroup;
        prof_begin(P_VOX_BWD, stream);
        k_vox_bwd<<<(unsigned)std::min<long long>(groups, 148 * 16), kVoxThreads, 0, stream>>>(rec, sorted, st, M,
                                                                                              gr, Tq, dvol, mom);
        prof_end(P_VOX_BWD, stream);
        note_launches(1);
    }
    if (parts & kVoxBwdChain) {
        Params P{mean, scale, quat, rho};
        prof_begin(P_VOX_CHAIN, stream);
        if (parts & kVoxBwdAssign)
            k_vox_chain<true><<<(unsigned)((M + 127) / 128), 128, 0, stream>>>(P, gr, M, mom, dmean, dscale, dquat,
                                                                              drho);
        else
            k_vox_chain<false><<<(unsigned)((M + 127) / 128), 128, 0, stream>>>(P, gr, M, mom, dmean, dscale, dquat,
                                                                               drho);
        prof_end(P_VOX_CHAIN, stream);
        note_launches(1);
    }
    return check_launch("r2g_voxelize_backward");
}
}  // namespace r2g

R2G_API r2g_status r2g_voxelize_backward(int64_t M, const float* mean, const float* scale, const float* quat,
                                         const float* rho, int32_t G, const r2g_grid* grids, float Q3,
                                         const float* dvol, float* dmean, float* dscale, float* dquat, float* drho,
                                         void* ws, size_t ws_bytes, r2g_stream stream) {
    return voxelize_backward_impl(M, mean, scale, quat, rho, G, grids, Q3, dvol, dmean, dscale, dquat, drho, ws,
                                  ws_bytes, stream, kVoxBwdMoments | kVoxBwdChain);
}

R2G_API r2g_status r2g_voxel_lists(int64_t M, int32_t G, const r2g_grid* grids, const void* ws, size_t ws_bytes,
                                   uint32_t* ranges_out, uint32_t* ids, int64_t capacity, int64_t* n_entries,
                                   r2g_stream stream) {
    Grids gr;
    r2g_status e = make_grids(G, grids, gr);
    if (e) return e;
    if (M < 1 || !ws || !ranges_out || !ids || !n_entries) return fail(R2G_E_INVAL, "bad argument");
    const VoxLayout L = vox_layout(M, gr);
    const long long cap = vox_capacity(L, ws_bytes);
    if (cap < 32) return fail(R2G_E_INVAL, "workspace of %zu bytes holds no list entries", ws_bytes);
    const VTail T = vox_tail(L, cap);
    const char* base = static_cast<const char*>(ws);
    WsStatus st;
    if (cudaMemcpyAsync(&st, base + L.status, sizeof(st), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "reading the workspace status failed");
    *n_entries = (int64_t)st.needed;
    if (st.status == R2G_E_CAPACITY) return fail(R2G_E_CAPACITY, "lists overflowed the workspace");
    if ((long long)st.n_keys > capacity) return fail(R2G_E_CAPACITY, "ids buffer too small");
    const uint64_t* sorted = vox_sorted(const_cast<char*>(base), L, T);
    if (cudaMemcpyAsync(ranges_out, base + L.ranges, 8 * (size_t)L.n_bricks, cudaMemcpyDeviceToDevice, stream) !=
            cudaSuccess ||
        (st.n_keys > 0 &&
         cudaMemcpy2DAsync(ids, 4, sorted, 8, 4, (size_t)st.n_keys, cudaMemcpyDeviceToDevice, stream) !=
             cudaSuccess) ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "copying the lists failed");
    return R2G_OK;
}
