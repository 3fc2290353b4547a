// fdk.cu -- the FDK initialisation of Sec. 4.1 on the GPU: the preliminary
// cone-beam reconstruction (Feldkamp-Davis-Kress: pre-weighting, ramp filtering
// of every detector row, distance-weighted back-projection), the seeded draw of M
// kernel positions among the voxels above the density threshold, and the
// nearest-neighbour scales.
//
// Filtering (one CTA per detector row).  R'(xi, eta) = R * L_SD / sqrt(L_SD^2 +
// xi^2 + eta^2) (cone beam); F(xi_n) = (1 / pitch_u) sum_m c_m R'(xi_{n-m}) with
// the Ram-Lak ramp in units of 1/tau^2 times the full-circle factor 1/2:
// c_0 = 1/8, c_m = -1/(2 pi^2 m^2) for odd m, 0 for even m.  The row sits in
// shared memory between zero margins (one skew word per 16 positions, so the
// lanes' windows fall in distinct banks); each thread produces 16 adjacent
// outputs and walks the odd taps eight at a time, reusing two sliding register
// windows (60 shared loads per 256 floating-point operations).
//
// Back-projection (one thread per (x, y) column and 16 consecutive z voxels).
// f(p) = dbeta sum_v w_v F_v(xi, eta), (xi, eta) = L_SD (u0, u1) / u2 and w_v =
// D_v L_SD / u2^2 (cone; D_v = t_v[2] is the source-to-isocentre depth), or
// (u0, u1) and 1 (parallel), u = W p + t; F is read by bilinear interpolation
// between pixel centres, samples outside the detector counting as zero.  The
// views' transforms are staged in shared memory 64 at a time.  When the view's
// rotation leaves u0 and u2 independent of z (rotation about the z axis, W's
// third column = (0, w12, 0)), the column's 16 voxels share xi, the column half
// of the bilinear weights and the distance weight.
//
// Selection.  Candidate voxel j (flat [z][y][x] index, vol[j] > tau) has the key
// SplitMix64(seed + (j + 1) * 0x9E3779B97F4A7C15); the M candidates with the
// smallest (key, j) are chosen.  The M-th smallest pair is found by radix select:
// four 16-bit digit passes over the key, then two over the index among the
// candidates whose key equals the threshold key (ties of 64-bit keys), each a
// histogram pass over the volume plus a one-CTA pass that finds the bin holding
// the wanted rank.  The chosen voxels are then written in increasing index order
// (per-block counts, one scan, an ordered block-wise compaction) as Gaussians:
// mean = voxel centre, identity rotation, rho = k * vol[j]; their cells are marked
// in an occupancy bit mask of the grid.
//
// Scales.  Each chosen position (one warp; the lanes share the (z, y) rows of a
// shell and read the occupancy mask a word at a time) searches the occupancy
// mask in cubic shells of growing Chebyshev radius r and keeps its three nearest
// other positions; once
// three are held and the third is no farther than (r + 1) * (smallest voxel
// edge), no unvisited cell can be nearer and the search stops.  The scale is the
// mean of the (up to) three distances; a position with no other position gets the
// smallest voxel edge.
#include <math.h>

#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr int kFiltJ = 16;    // outputs per thread (a power of two: see skew())
constexpr int kFiltS = 8;     // odd taps per window step
constexpr int kBpZ = 16;      // voxels per back-projection thread (along z)
constexpr int kBpViews = 64;  // views staged in shared memory at a time
constexpr int kSelDigits = 16;
constexpr int kSelBins = 1 << kSelDigits;
constexpr int kSelBlocks = 148 * 6;   // fixed grid of the selection passes (<= 1024: one scan CTA)
constexpr int kKnnMaxR = 4096;
constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------------ filtering

// Shared-memory slot of padded row position k: one skew word per kFiltJ, so that
// lanes whose windows start kFiltJ positions apart are kFiltJ + 1 (odd) slots
// apart and hit distinct banks.
__device__ __forceinline__ int skew(int k) { return k + k / kFiltJ; }

__global__ void __launch_bounds__(256) k_fdk_filter(const float* __restrict__ proj, float* __restrict__ filt, int H,
                                                    int W, int cone, float L_SD, float pu, float pv, float ou,
                                                    float ov, float inv_pu) {
    extern __shared__ float sm[];
    // zero margin on each side of the row, P = 15 (mod 16): with outputs n0 a
    // multiple of kFiltJ = 16 and taps m0 = 1 (mod 16), both windows below start at
    // multiples of 16, so slot(start + i) = slot(start) + i + i / 16
    const int P = ((W + 32 + 15) / 16) * 16 + 15;
    const int n_row = W + 2 * P;           // padded row positions
    float* tap = sm + skew(n_row) + 8;     // tap[m], m = 0 .. W + 2 kFiltS + 1 (0 beyond W - 1)
    const long long r = blockIdx.x;
    const int rr = (int)(r % H);
    const float* src = proj + r * W;
    const float eta = ((float)rr + 0.5f - 0.5f * (float)H) * pv + ov;
    for (int k = threadIdx.x; k < n_row; k += blockDim.x) {
        const int c = k - P;
        float x = 0.f;
        if (c >= 0 && c < W) {
            x = src[c];
            if (cone) {
                const float xi = ((float)c + 0.5f - 0.5f * (float)W) * pu + ou;
                x *= L_SD * __frsqrt_rn(L_SD * L_SD + xi * xi + eta * eta);
            }
        }
        sm[skew(k)] = x;
    }
    const float kInv2Pi2 = 0.05066059182116889f;  // 1 / (2 pi^2)
    for (int m = threadIdx.x; m < W + 2 * kFiltS + 2; m += blockDim.x)
        tap[m] = (m & 1) && m < W ? -kInv2Pi2 / ((float)m * (float)m) : 0.f;
    __syncthreads();
    const int n0 = threadIdx.x * kFiltJ;
    if (n0 >= W) return;
    float acc[kFiltJ];
#pragma unroll
    for (int j = 0; j < kFiltJ; ++j) acc[j] = 0.125f * sm[skew(P + n0 + j)];
    // taps m0, m0 + 2, ..., m0 + 2(S-1):
    //   left  R[n0 + j - m0 - 2s] = L[j - 2s + 2(S-1)],  L[i] = R[n0 - m0 - 2(S-1) + i]
    //   right R[n0 + j + m0 + 2s] = Rw[j + 2s],            Rw[i] = R[n0 + m0 + i]
    // padded starts: P + n0 - m0 - 14 and P + n0 + m0, both multiples of 16
    constexpr int NW = kFiltJ + 2 * (kFiltS - 1);
    static_assert(kFiltJ == 16 && kFiltS == 8, "window alignment assumes 16 outputs and 8 taps per step");
    const float* lp = sm + skew(P + n0 - 15);   // left window start for m0 = 1
    const float* rp = sm + skew(P + n0 + 1);    // right window start for m0 = 1
    for (int m0 = 1; m0 < W; m0 += 2 * kFiltS, lp -= kFiltJ + 1, rp += kFiltJ + 1) {
        float L[NW], Rw[NW], c[kFiltS];
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            L[i] = lp[i + i / 16];
            Rw[i] = rp[i + i / 16];
        }
#pragma unroll
        for (int s2 = 0; s2 < kFiltS; ++s2) c[s2] = tap[m0 + 2 * s2];
#pragma unroll
        for (int s2 = 0; s2 < kFiltS; ++s2)
#pragma unroll
            for (int j = 0; j < kFiltJ; ++j)
                acc[j] = fmaf(c[s2], L[j - 2 * s2 + 2 * (kFiltS - 1)] + Rw[j + 2 * s2], acc[j]);
    }
    float* dst = filt + r * W;
#pragma unroll
    for (int j = 0; j < kFiltJ; ++j)
        if (n0 + j < W) dst[n0 + j] = acc[j] * inv_pu;
}

// ------------------------------------------------------------------ back-projection

struct BpCam {
    int H, W;
    float L_SD, inv_pu, inv_pv, cu, cv, near_plane;  // cu = W/2 - 1/2 - off_u / pitch_u (columns), rows alike
};

__device__ __forceinline__ float bilerp(const float* __restrict__ img, int H, int W, float xc, float yc) {
    xc = fminf(fmaxf(xc, -2.f), (float)W + 1.f);
    yc = fminf(fmaxf(yc, -2.f), (float)H + 1.f);
    const float fx = floorf(xc), fy = floorf(yc);
    const int x0 = (int)fx, y0 = (int)fy;
    const float ax = xc - fx, ay = yc - fy;
    const bool xa = x0 >= 0 && x0 < W, xb = x0 >= -1 && x0 < W - 1;
    const bool ya = y0 >= 0 && y0 < H, yb = y0 >= -1 && y0 < H - 1;
    const float* p = img + (long long)y0 * W + x0;
    const float v00 = (ya && xa) ? __ldg(p) : 0.f;
    const float v01 = (ya && xb) ? __ldg(p + 1) : 0.f;
    const float v10 = (yb && xa) ? __ldg(p + W) : 0.f;
    const float v11 = (yb && xb) ? __ldg(p + W + 1) : 0.f;
    const float top = fmaf(ax, v01 - v00, v00);
    const float bot = fmaf(ax, v11 - v10, v10);
    return fmaf(ay, bot - top, top);
}

// Column half of the bilinear read, shared by the voxels of a column whose
// detector column does not change along z.
struct ColW {
    int x0;
    float ax;
    bool xa, xb;
};

__device__ __forceinline__ ColW col_weights(float xc, int W) {
    xc = fminf(fmaxf(xc, -2.f), (float)W + 1.f);
    const float fx = floorf(xc);
    ColW c;
    c.x0 = (int)fx;
    c.ax = xc - fx;
    c.xa = c.x0 >= 0 && c.x0 < W;
    c.xb = c.x0 >= -1 && c.x0 < W - 1;
    return c;
}

__device__ __forceinline__ float bilerp_col(const float* __restrict__ img, int H, int W, const ColW& c, float yc) {
    yc = fminf(fmaxf(yc, -2.f), (float)H + 1.f);
    const float fy = floorf(yc);
    const int y0 = (int)fy;
    const float ay = yc - fy;
    const bool ya = y0 >= 0 && y0 < H, yb = y0 >= -1 && y0 < H - 1;
    const float* p = img + (long long)y0 * W + c.x0;
    const float v00 = (ya && c.xa) ? __ldg(p) : 0.f;
    const float v01 = (ya && c.xb) ? __ldg(p + 1) : 0.f;
    const float v10 = (yb && c.xa) ? __ldg(p + W) : 0.f;
    const float v11 = (yb && c.xb) ? __ldg(p + W + 1) : 0.f;
    const float top = fmaf(c.ax, v01 - v00, v00);
    const float bot = fmaf(c.ax, v11 - v10, v10);
    return fmaf(ay, bot - top, top);
}

template <bool CONE>
__global__ void __launch_bounds__(256) k_fdk_bp(const float* __restrict__ filt, const float* __restrict__ views, int V,
                                                BpCam cam, float3 org, float3 vs, int X, int Y, int Z, float dbeta,
                                                float* __restrict__ vol) {
    __shared__ float sv[kBpViews][13];
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z0 = blockIdx.z * kBpZ;
    const float px = org.x + ((float)x + 0.5f) * vs.x;
    const float py = org.y + ((float)y + 0.5f) * vs.y;
    const float pz = org.z + ((float)z0 + 0.5f) * vs.z;
    float acc[kBpZ];
#pragma unroll
    for (int j = 0; j < kBpZ; ++j) acc[j] = 0.f;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const long long img_px = (long long)cam.H * cam.W;
    for (int v0 = 0; v0 < V; v0 += kBpViews) {
        const int nv = min(kBpViews, V - v0);
        __syncthreads();
        for (int k = tid; k < nv * 12; k += 256) sv[k / 12][k % 12] = views[(long long)v0 * 12 + k];
        __syncthreads();
        if (x >= X || y >= Y) continue;
        for (int vv = 0; vv < nv; ++vv) {
            const float* w = sv[vv];
            const float* img = filt + (long long)(v0 + vv) * img_px;
            float u0 = fmaf(w[0], px, fmaf(w[1], py, fmaf(w[2], pz, w[9])));
            float u1 = fmaf(w[3], px, fmaf(w[4], py, fmaf(w[5], pz, w[10])));
            float u2 = fmaf(w[6], px, fmaf(w[7], py, fmaf(w[8], pz, w[11])));
            const float d0 = w[2] * vs.z, d1 = w[5] * vs.z, d2 = w[8] * vs.z;
            if (CONE) {
                const float DL = w[11] * cam.L_SD;
                if (w[2] == 0.f && w[8] == 0.f) {
                    // u0, u2 constant along the column: one reciprocal, one weight
                    if (u2 > cam.near_plane) {
                        const float inv = 1.0f / u2;
                        const ColW cw = col_weights(fmaf(cam.L_SD * u0 * inv, cam.inv_pu, cam.cu), cam.W);
                        const float wt = DL * inv * inv;
                        const float ys = cam.L_SD * inv * cam.inv_pv;
#pragma unroll
                        for (int j = 0; j < kBpZ; ++j) {
                            const float yc = fmaf(u1 + (float)j * d1, ys, cam.cv);
                            acc[j] = fmaf(wt, bilerp_col(img, cam.H, cam.W, cw, yc), acc[j]);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < kBpZ; ++j) {
                        if (u2 > cam.near_plane) {
                            const float inv = 1.0f / u2;
                            const float xc = fmaf(cam.L_SD * u0 * inv, cam.inv_pu, cam.cu);
                            const float yc = fmaf(cam.L_SD * u1 * inv, cam.inv_pv, cam.cv);
                            acc[j] = fmaf(DL * inv * inv, bilerp(img, cam.H, cam.W, xc, yc), acc[j]);
                        }
                        u0 += d0;
                        u1 += d1;
                        u2 += d2;
                    }
                }
            } else if (w[2] == 0.f) {
                const ColW cw = col_weights(fmaf(u0, cam.inv_pu, cam.cu), cam.W);
#pragma unroll
                for (int j = 0; j < kBpZ; ++j)
                    acc[j] += bilerp_col(img, cam.H, cam.W, cw, fmaf(u1 + (float)j * d1, cam.inv_pv, cam.cv));
            } else {
#pragma unroll
                for (int j = 0; j < kBpZ; ++j) {
                    const float xc = fmaf(u0 + (float)j * d0, cam.inv_pu, cam.cu);
                    const float yc = fmaf(u1 + (float)j * d1, cam.inv_pv, cam.cv);
                    acc[j] += bilerp(img, cam.H, cam.W, xc, yc);
                }
            }
        }
    }
    if (x >= X || y >= Y) return;
#pragma unroll
    for (int j = 0; j < kBpZ; ++j)
        if (z0 + j < Z) vol[((long long)(z0 + j) * Y + y) * X + x] = dbeta * acc[j];
}

// ------------------------------------------------------------------ selection

struct SelState {
    unsigned long long need;     // rank still wanted inside the current prefix
    unsigned long long kprefix;  // key bits fixed so far (top 16 * pass bits)
    unsigned long long n_cand;   // candidates (pass 0 total)
    unsigned int iprefix;        // index bits fixed so far (index passes)
    unsigned int take_all;       // 1: at most M candidates, all are taken
    unsigned long long n_sel;    // positions written
    unsigned long long pad[3];
};
static_assert(sizeof(SelState) == 64, "selection state is 64 bytes");

struct SelArgs {
    const float* vol;
    long long n;
    float tau;
    unsigned long long seed;
};

__device__ __forceinline__ bool candidate(const SelArgs& a, long long j, unsigned long long* key) {
    if (!(a.vol[j] > a.tau)) return false;
    *key = splitmix64(a.seed + (unsigned long long)(j + 1) * kGolden);
    return true;
}

// pass 0..3: 16-bit digits of the key (most significant first) among candidates
// whose key matches the prefix fixed so far; pass 4, 5: digits of the index among
// candidates whose key equals the threshold key.
__global__ void __launch_bounds__(256) k_sel_hist(SelArgs a, int pass, const SelState* __restrict__ st,
                                                  unsigned int* __restrict__ hist) {
    if (st->take_all) return;
    const unsigned long long kp = st->kprefix;
    const unsigned int ip = st->iprefix;
    for (long long j = (long long)blockIdx.x * 256 + threadIdx.x; j < a.n; j += (long long)gridDim.x * 256) {
        unsigned long long key;
        if (!candidate(a, j, &key)) continue;
        unsigned int digit;
        if (pass < 4) {
            const int hi = 64 - 16 * pass;  // bits above `hi` must match the prefix
            if (pass > 0 && (key >> hi) != kp) continue;
            digit = (unsigned int)(key >> (hi - 16)) & 0xffffu;
        } else {
            if (key != kp) continue;
            const unsigned int ju = (unsigned int)j;
            if (pass == 5 && (ju >> 16) != ip) continue;
            digit = pass == 4 ? (ju >> 16) : (ju & 0xffffu);
        }
        atomicAdd(&hist[digit], 1u);
    }
}

// One CTA of 1024 threads: the bin of the wanted rank; the prefix grows by that
// digit and the rank becomes the rank inside the bin.  Clears the histogram.
// Warp w owns bins [w * 2048, (w + 1) * 2048), read 32 at a time (coalesced).
__global__ void __launch_bounds__(1024) k_sel_find(int pass, long long M, SelState* __restrict__ st,
                                                   unsigned int* __restrict__ hist) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long total_s;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int kPerWarp = kSelBins / 32;
    const unsigned int* h = hist + warp * kPerWarp;
    unsigned long long mine = 0;
    for (int c = lane; c < kPerWarp; c += 32) mine += h[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) wsum[warp] = mine;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long s = wsum[lane];
        unsigned long long incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        wsum[lane] = incl - s;  // candidates in the warps before
        if (lane == 31) total_s = incl;
    }
    __syncthreads();
    const unsigned long long total = total_s;
    const bool take_all = pass == 0 && total <= (unsigned long long)M;
    const unsigned long long need = pass == 0 ? (unsigned long long)M : st->need;
    __syncthreads();
    if (pass == 0 && t == 0) {  // st->need is written only by the warp that finds the bin
        st->n_cand = total;
        st->take_all = take_all ? 1u : 0u;
    }
    const unsigned long long before = wsum[warp];
    if (!take_all && need > before && need <= before + mine) {
        // this warp holds the bin: walk its chunks of 32 bins in order
        unsigned long long c0 = before;
        for (int c = 0; c < kPerWarp; c += 32) {
            const unsigned int v = h[c + lane];
            unsigned long long incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned long long lo = c0 + incl - v;
            if (need > lo && need <= lo + v) {
                const unsigned int digit = (unsigned int)(warp * kPerWarp + c + lane);
                st->need = need - lo;
                if (pass < 4)
                    st->kprefix = (st->kprefix << 16) | digit;
                else
                    st->iprefix = pass == 4 ? digit : ((st->iprefix << 16) | digit);
            }
            c0 += __shfl_sync(0xffffffffu, incl, 31);
            if (c0 >= need) break;
        }
    }
    __syncthreads();
    for (int i = t; i < kSelBins; i += 1024) hist[i] = 0u;
}

__device__ __forceinline__ bool selected(const SelArgs& a, const SelState& st, long long j) {
    unsigned long long key;
    if (!candidate(a, j, &key)) return false;
    if (st.take_all) return true;
    return key < st.kprefix || (key == st.kprefix && (unsigned int)j <= st.iprefix);
}

__device__ __forceinline__ void block_range(long long n, long long* lo, long long* hi) {
    const long long per = ((n + gridDim.x - 1) / gridDim.x + 255) / 256 * 256;
    *lo = min(n, (long long)blockIdx.x * per);
    *hi = min(n, *lo + per);
}

__global__ void __launch_bounds__(256) k_sel_count(SelArgs a, const SelState* __restrict__ st,
                                                   unsigned int* __restrict__ counts) {
    __shared__ unsigned int red[8];
    const SelState s = *st;
    long long lo, hi;
    block_range(a.n, &lo, &hi);
    unsigned int c = 0;
    for (long long j = lo + threadIdx.x; j < hi; j += 256) c += selected(a, s, j) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0;
        for (int w = 0; w < 8; ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}

// One CTA: exclusive scan of the per-block counts (in place) and the total.
__global__ void __launch_bounds__(1024) k_sel_scan(unsigned int* __restrict__ counts, int nb, SelState* __restrict__ st,
                                                   long long* __restrict__ n_out) {
    __shared__ unsigned int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned int v = t < nb ? counts[t] : 0u;
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
        if (lane == 31) {
            st->n_sel = incl;
            *n_out = (long long)incl;
        }
    }
    __syncthreads();
    if (t < nb) counts[t] = wsum[warp] + x - v;
}

struct GridF {
    float ox, oy, oz, vx, vy, vz;
    int X, Y, Z;
};

__global__ void __launch_bounds__(256) k_sel_write(SelArgs a, const SelState* __restrict__ st,
                                                   const unsigned int* __restrict__ offsets, GridF g, float k,
                                                   float* __restrict__ mean, float* __restrict__ quat,
                                                   float* __restrict__ rho, unsigned int* __restrict__ sel_idx,
                                                   unsigned int* __restrict__ occ) {
    __shared__ uint32_t scan_sm[8];
    const SelState s = *st;
    long long lo, hi;
    block_range(a.n, &lo, &hi);
    unsigned int base = offsets[blockIdx.x];
    for (long long c0 = lo; c0 < hi; c0 += 256) {
        const long long j = c0 + threadIdx.x;
        const bool on = j < hi && selected(a, s, j);
        uint32_t tot;
        const uint32_t off = block_exclusive_scan_256(on ? 1u : 0u, scan_sm, &tot);
        if (on) {
            const unsigned int o = base + off;
            const long long XY = (long long)g.X * g.Y;
            const int z = (int)(j / XY), y = (int)((j / g.X) % g.Y), x = (int)(j % g.X);
            mean[3ll * o + 0] = g.ox + ((float)x + 0.5f) * g.vx;
            mean[3ll * o + 1] = g.oy + ((float)y + 0.5f) * g.vy;
            mean[3ll * o + 2] = g.oz + ((float)z + 0.5f) * g.vz;
            reinterpret_cast<float4*>(quat)[o] = make_float4(1.f, 0.f, 0.f, 0.f);
            rho[o] = k * a.vol[j];
            sel_idx[o] = (unsigned int)j;
            atomicOr(&occ[j >> 5], 1u << (j & 31));
        }
        base += tot;
    }
}

// The three smallest squared distances so far, ascending (+inf while fewer).
__device__ __forceinline__ void keep3(float d2, float& b0, float& b1, float& b2) {
    if (d2 < b2) {
        b2 = d2;
        if (b2 < b1) {
            const float t = b1;
            b1 = b2;
            b2 = t;
        }
        if (b1 < b0) {
            const float t = b0;
            b0 = b1;
            b1 = t;
        }
    }
}

// Occupied cells among flat bit indices [lo, hi] of one grid row (rowj = flat
// index of the row's x = 0 cell), folded into the three nearest.
__device__ __forceinline__ void scan_row(const unsigned int* __restrict__ occ, long long lo, long long hi,
                                         long long rowj, int cx, float vx, float eyz2, float& b0, float& b1,
                                         float& b2) {
    for (long long w = lo >> 5; w <= (hi >> 5); ++w) {
        unsigned int bits = __ldg(&occ[w]);
        const long long wb = w << 5;
        if (wb < lo) bits &= ~0u << (int)(lo - wb);
        if (hi - wb < 31) bits &= (2u << (int)(hi - wb)) - 1u;
        while (bits) {
            const int t = __ffs(bits) - 1;
            bits &= bits - 1u;
            const float ex = (float)((int)(wb + t - rowj) - cx) * vx;
            keep3(fmaf(ex, ex, eyz2), b0, b1, b2);
        }
    }
}

// The three smallest of the warp's per-lane lists (every lane gets them).
__device__ __forceinline__ void warp_top3(float b0, float b1, float b2, float out[3]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float m = b0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        out[k] = m;
        const unsigned int owner = __ballot_sync(0xffffffffu, b0 == m);
        if (lane == __ffs(owner) - 1) {
            b0 = b1;
            b1 = b2;
            b2 = INFINITY;
        }
    }
}

// One warp per chosen position; the lanes share each shell's (z, y) rows.
__global__ void __launch_bounds__(256) k_knn3(const unsigned int* __restrict__ sel_idx,
                                              const SelState* __restrict__ st, const unsigned int* __restrict__ occ,
                                              GridF g, float vmin, float* __restrict__ scale) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= (long long)st->n_sel) return;  // whole warps
    const long long j = sel_idx[i];
    const long long XY = (long long)g.X * g.Y;
    const int cz = (int)(j / XY), cy = (int)((j / g.X) % g.Y), cx = (int)(j % g.X);
    float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY;
    float top[3];
    const int rmax = min(kKnnMaxR, max(g.X, max(g.Y, g.Z)));
    for (int r = 1; r <= rmax; ++r) {
        const int side = 2 * r + 1;
        for (int q = lane; q < side * side; q += 32) {
            const int dz = q / side - r, dy = q % side - r;
            const int z = cz + dz, y = cy + dy;
            if (z < 0 || z >= g.Z || y < 0 || y >= g.Y) continue;
            const float ez = (float)dz * g.vz, ey = (float)dy * g.vy;
            const float eyz2 = fmaf(ey, ey, ez * ez);
            const long long rowj = ((long long)z * g.Y + y) * g.X;
            if (dz == -r || dz == r || dy == -r || dy == r) {
                scan_row(occ, rowj + max(cx - r, 0), rowj + min(cx + r, g.X - 1), rowj, cx, g.vx, eyz2, b0, b1, b2);
            } else {
                if (cx - r >= 0) scan_row(occ, rowj + cx - r, rowj + cx - r, rowj, cx, g.vx, eyz2, b0, b1, b2);
                if (cx + r < g.X) scan_row(occ, rowj + cx + r, rowj + cx + r, rowj, cx, g.vx, eyz2, b0, b1, b2);
            }
        }
        warp_top3(b0, b1, b2, top);
        const float reach = (float)(r + 1) * vmin;
        if (top[2] <= reach * reach) break;                     // no unvisited cell is nearer
        if (r >= g.X && r >= g.Y && r >= g.Z) break;             // the whole grid has been visited
    }
    if (lane != 0) return;
    float s = vmin;
    if (top[2] < INFINITY)
        s = (sqrtf(top[0]) + sqrtf(top[1]) + sqrtf(top[2])) / 3.f;
    else if (top[1] < INFINITY)
        s = 0.5f * (sqrtf(top[0]) + sqrtf(top[1]));
    else if (top[0] < INFINITY)
        s = sqrtf(top[0]);
    scale[3 * i + 0] = s;
    scale[3 * i + 1] = s;
    scale[3 * i + 2] = s;
}

// ------------------------------------------------------------------ host side

struct InitLayout {
    size_t state, hist, counts, occ, sel, total;
};

InitLayout init_layout(long long n_vox, long long M) {
    Layout L;
    InitLayout o;
    o.state = L.take(sizeof(SelState));
    o.hist = L.take(sizeof(unsigned int) * kSelBins);
    o.counts = L.take(sizeof(unsigned int) * kSelBlocks);
    o.occ = L.take(sizeof(unsigned int) * (size_t)((n_vox + 31) / 32));
    o.sel = L.take(sizeof(unsigned int) * (size_t)M);
    o.total = L.off;
    return o;
}

r2g_status check_grid(const r2g_grid* g, long long* n_vox) {
    if (!g) return fail(R2G_E_INVAL, "grid is NULL");
    for (int a = 0; a < 3; ++a) {
        if (g->dims[a] < 1 || g->dims[a] > 4096) return fail(R2G_E_INVAL, "grid dims must be 1..4096");
        if (!(g->voxel[a] > 0.f)) return fail(R2G_E_INVAL, "voxel size must be > 0");
    }
    *n_vox = (long long)g->dims[0] * g->dims[1] * g->dims[2];
    if (*n_vox >= (1ll << 31)) return fail(R2G_E_INVAL, "grid has 2^31 voxels or more");
    return R2G_OK;
}

r2g_status check_cam(const r2g_camera* cam) {
    if (!cam) return fail(R2G_E_INVAL, "camera is NULL");
    if (cam->beam != 0 && cam->beam != 1) return fail(R2G_E_INVAL, "beam must be 0 or 1");
    if (cam->H < 1 || cam->W < 1 || cam->H > 32768 || cam->W > 32768) return fail(R2G_E_INVAL, "bad detector size");
    if (!(cam->pitch_u > 0.f) || !(cam->pitch_v > 0.f)) return fail(R2G_E_INVAL, "pitch must be > 0");
    if (cam->beam == 1 && !(cam->L_SD > 0.f)) return fail(R2G_E_INVAL, "cone beam needs L_SD > 0");
    return R2G_OK;
}

GridF gridf(const r2g_grid* g) {
    return GridF{g->origin[0], g->origin[1], g->origin[2], g->voxel[0], g->voxel[1], g->voxel[2],
                 g->dims[0],   g->dims[1],   g->dims[2]};
}

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API r2g_status r2g_fdk_filter(int32_t V, const r2g_camera* cam, const float* proj, float* filt,
                                  r2g_stream stream) {
    if (r2g_status e = check_cam(cam)) return e;
    if (V < 1 || V > 65535) return fail(R2G_E_INVAL, "V must be 1..65535");
    if (cam->W > 8192) return fail(R2G_E_INVAL, "the FDK filter takes at most 8192 detector columns");
    if (!proj || !filt) return fail(R2G_E_INVAL, "NULL device pointer");
    if (proj == filt) return fail(R2G_E_INVAL, "proj and filt must not alias");
    const int W = cam->W;
    const int threads = ((W + kFiltJ - 1) / kFiltJ + 31) / 32 * 32;
    const int P = ((W + 32 + 15) / 16) * 16 + 15;  // as in the kernel
    const int n_row = W + 2 * P;
    const size_t smem = sizeof(float) * (size_t)(n_row + n_row / kFiltJ + 8 + W + 2 * kFiltS + 2);
    // the row's shared memory may exceed the 48 KB default: opt in once per device
    // (idempotent, so racing first calls are harmless)
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_fdk_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess)
            return fail(R2G_E_CUDA, "r2g_fdk_filter: shared memory attribute (%s)",
                        cudaGetErrorString(cudaGetLastError()));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    prof_begin(P_FDK_FILTER, stream);
    k_fdk_filter<<<(unsigned)((long long)V * cam->H), threads, smem, stream>>>(
        proj, filt, cam->H, W, cam->beam, cam->L_SD, cam->pitch_u, cam->pitch_v, cam->off_u, cam->off_v,
        1.0f / cam->pitch_u);
    prof_end(P_FDK_FILTER, stream);
    note_launches(1);
    return check_launch("r2g_fdk_filter");
}

R2G_API r2g_status r2g_fdk_backproject(int32_t V, const float* views, const r2g_camera* cam, const float* filt,
                                       const r2g_grid* grid, float dbeta, float* vol, r2g_stream stream) {
    if (r2g_status e = check_cam(cam)) return e;
    long long n_vox;
    if (r2g_status e = check_grid(grid, &n_vox)) return e;
    if (V < 1 || V > 65535) return fail(R2G_E_INVAL, "V must be 1..65535");
    if (!views || !filt || !vol) return fail(R2G_E_INVAL, "NULL device pointer");
    BpCam c;
    c.H = cam->H;
    c.W = cam->W;
    c.L_SD = cam->L_SD;
    c.inv_pu = 1.0f / cam->pitch_u;
    c.inv_pv = 1.0f / cam->pitch_v;
    c.cu = 0.5f * (float)cam->W - 0.5f - cam->off_u * c.inv_pu;
    c.cv = 0.5f * (float)cam->H - 0.5f - cam->off_v * c.inv_pv;
    c.near_plane = cam->near_plane;
    const int X = grid->dims[0], Y = grid->dims[1], Z = grid->dims[2];
    const dim3 blk(32, 8);
    const dim3 grd((unsigned)((X + 31) / 32), (unsigned)((Y + 7) / 8), (unsigned)((Z + kBpZ - 1) / kBpZ));
    const float3 org = make_float3(grid->origin[0], grid->origin[1], grid->origin[2]);
    const float3 vs = make_float3(grid->voxel[0], grid->voxel[1], grid->voxel[2]);
    prof_begin(P_FDK_BP, stream);
    if (cam->beam == 1)
        k_fdk_bp<true><<<grd, blk, 0, stream>>>(filt, views, V, c, org, vs, X, Y, Z, dbeta, vol);
    else
        k_fdk_bp<false><<<grd, blk, 0, stream>>>(filt, views, V, c, org, vs, X, Y, Z, dbeta, vol);
    prof_end(P_FDK_BP, stream);
    note_launches(1);
    return check_launch("r2g_fdk_backproject");
}

R2G_API size_t r2g_init_workspace_size(const r2g_grid* grid, int64_t M) {
    long long n_vox;
    if (check_grid(grid, &n_vox) || M < 1) return 0;
    return init_layout(n_vox, M).total;
}

R2G_API r2g_status r2g_init_gaussians(const float* vol, const r2g_grid* grid, float tau, int64_t M, uint64_t seed,
                                      float k, float* mean, float* scale, float* quat, float* rho, int64_t* n_out,
                                      void* ws, size_t ws_bytes, r2g_stream stream) {
    long long n_vox;
    if (r2g_status e = check_grid(grid, &n_vox)) return e;
    if (M < 1 || M >= (1ll << 31)) return fail(R2G_E_INVAL, "M must be 1 .. 2^31 - 1");
    if (!vol || !mean || !scale || !quat || !rho || !n_out || !ws) return fail(R2G_E_INVAL, "NULL device pointer");
    if (reinterpret_cast<uintptr_t>(quat) % 16) return fail(R2G_E_INVAL, "quat must be 16-byte aligned");
    const InitLayout L = init_layout(n_vox, M);
    if (ws_bytes < L.total) return fail(R2G_E_INVAL, "workspace too small: %zu < %zu", ws_bytes, L.total);
    char* base = static_cast<char*>(ws);
    SelState* st = reinterpret_cast<SelState*>(base + L.state);
    unsigned int* hist = reinterpret_cast<unsigned int*>(base + L.hist);
    unsigned int* counts = reinterpret_cast<unsigned int*>(base + L.counts);
    unsigned int* occ = reinterpret_cast<unsigned int*>(base + L.occ);
    unsigned int* sel = reinterpret_cast<unsigned int*>(base + L.sel);
    // state, histogram (contiguous after the state) and occupancy start at zero
    cudaMemsetAsync(base, 0, L.counts, stream);
    cudaMemsetAsync(occ, 0, sizeof(unsigned int) * (size_t)((n_vox + 31) / 32), stream);
    const SelArgs a{vol, n_vox, tau, (unsigned long long)seed};
    prof_begin(P_INIT_SELECT, stream);
    for (int pass = 0; pass < 6; ++pass) {
        k_sel_hist<<<kSelBlocks, 256, 0, stream>>>(a, pass, st, hist);
        k_sel_find<<<1, 1024, 0, stream>>>(pass, (long long)M, st, hist);
    }
    k_sel_count<<<kSelBlocks, 256, 0, stream>>>(a, st, counts);
    k_sel_scan<<<1, 1024, 0, stream>>>(counts, kSelBlocks, st, reinterpret_cast<long long*>(n_out));
    const GridF g = gridf(grid);
    k_sel_write<<<kSelBlocks, 256, 0, stream>>>(a, st, counts, g, k, mean, quat, rho, sel, occ);
    prof_end(P_INIT_SELECT, stream);
    const float vmin = fminf(g.vx, fminf(g.vy, g.vz));
    prof_begin(P_INIT_KNN, stream);
    k_knn3<<<(unsigned)((M * 32 + 255) / 256), 256, 0, stream>>>(sel, st, occ, g, vmin, scale);
    prof_end(P_INIT_KNN, stream);
    note_launches(16);
    return check_launch("r2g_init_gaussians");
}
