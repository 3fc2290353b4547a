// loss.cu -- the training losses of Eq. 8 on sm_103a, forward and gradient fused.
//
// Projection loss L1 + lambda_ssim (1 - SSIM) over [V][H][W]:
//   k_ssim        one CTA per 32x32 output tile of one view: render x and
//                 measurement y staged with a 10-pixel halo (zeros outside the
//                 image), the 11-tap Gaussian window applied separably to x, y,
//                 xx, yy, xy, each pixel's SSIM term S and its derivatives with
//                 respect to the local moments (dS/dmu_x, dS/dE_xx, dS/dE_xy) on
//                 the tile plus a 5-pixel halo, those maps filtered again with
//                 the window (the adjoint of a zero-padded symmetric filter is
//                 itself) and combined with x, y and the L1 sign into d loss /
//                 d render; the last CTA to finish sums the per-tile partials
//                 in a fixed order into the loss (deterministic).
//   k_tv_sum      (TV) one CTA sums the per-CTA partials in a fixed order.
// 3D TV: k_tv3d forms each voxel's gradient from its six neighbours and a CTA
// partial of the loss; k_tv_sum sums the partials (k_finalize for the isotropic form).
#include <math.h>

#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr int kT = 32;            // output tile edge
constexpr int kR = 5;             // window radius
constexpr int kM = kT + 2 * kR;   // edge of the SSIM-derivative region (tile + halo)
constexpr int kS = kT + 4 * kR;   // edge of the staged input region
constexpr int kSsimThreads = 512;

// Normalised 1D Gaussian window (sigma 1.5), passed by value to each launch.
struct Win {
    float w[11];
};

constexpr float kC1 = 1e-4f;      // (0.01 L)^2, L = 1
constexpr float kC2 = 9e-4f;      // (0.03 L)^2

struct SsimSmem {
    float sx[kS][kS + 1], sy[kS][kS + 1];  // render x and measurement y, zeros outside the image
    union {
        float h[5][kS][kM + 1];            // horizontally filtered x, y, xx, yy, xy
        float g[3][kM][kT + 1];            // horizontally filtered derivative maps
    } u;
    float d[3][kM][kM + 1];                // dS/dmu_x, dS/dE_xx, dS/dE_xy (zero outside the image)
    float red[2][kSsimThreads / 32];
    int last;
};

// The thread that publishes the CTA's partial sums: one of the threads that write
// no d loss / d render (the last pass uses threads 0 .. kT * kT / 4 - 1), so its
// release fence does not wait for gradient stores.
constexpr int kArriveThread = kSsimThreads - 1;
static_assert(kArriveThread >= kT * kT / 4, "the arriving thread writes no gradient");

// Stage one image's tile plus its 10-pixel halo into dst (zeros outside the image).
// vec4: aligned float4 groups of columns TX - 12 .. TX + 43, the outer two on each
// side dropped, every load issued before any store; else one float per thread.
__device__ __forceinline__ void stage_tile(float (*dst)[kS + 1], const float* __restrict__ img, int TY, int TX,
                                           int H, int W, int tid, int vec4) {
    if (vec4) {
        constexpr int G = (kS + 4 + 3) / 4;          // float4 groups per staged row (14)
        constexpr int N = kS * G;
        constexpr int IT = (N + kSsimThreads - 1) / kSsimThreads;
        float4 val[IT];
#pragma unroll
        for (int t = 0; t < IT; ++t) {
            const int k = tid + t * kSsimThreads;
            val[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < N) {
                const int r = k / G, g = k - r * G;
                const int gy = TY - 2 * kR + r, gx = TX - 2 * kR - 2 + 4 * g;  // gx % 4 == 0
                if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                    val[t] = __ldg(reinterpret_cast<const float4*>(img + (size_t)gy * W + gx));
            }
        }
#pragma unroll
        for (int t = 0; t < IT; ++t) {
            const int k = tid + t * kSsimThreads;
            if (k < N) {
                const int r = k / G, g = k - r * G;
                const int c = 4 * g - 2;             // staged column of the group's first element
                const float e[4] = {val[t].x, val[t].y, val[t].z, val[t].w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c + q >= 0 && c + q < kS) dst[r][c + q] = e[q];
            }
        }
    } else {
        for (int k = tid; k < kS * kS; k += kSsimThreads) {
            const int r = k / kS, c = k - r * kS;
            const int gy = TY - 2 * kR + r, gx = TX - 2 * kR + c;
            dst[r][c] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? img[(size_t)gy * W + gx] : 0.f;
        }
    }
}

// One CTA per 32 x 32 output tile of one view.  x and y are staged with a
// 10-pixel halo; the windowed moments and each pixel's SSIM term S and its
// derivatives with respect to mu_x, E_xx and E_xy are formed on the tile plus a
// 5-pixel halo (zero outside the image, whose pixels the mean leaves out), from the
// moments of both images shifted by one constant per CTA; those
// derivative maps are filtered again with the window (the adjoint of a
// zero-padded symmetric filter is itself) and combined with x, y and the L1 sign
// into d loss / d render.  Per-tile sums of 1 - S and |x - y| go to `partials`;
// the last CTA to finish (arrival counter cleared before the launch) sums them in
// tile order into the loss (FP32 trees in a fixed order; 1 - S is summed rather
// than S so that no cancellation is left when SSIM nears 1).  meas_sel (optional,
// device): view v of the batch is compared with measurement meas_sel[v] of y.
// vec4: W % 4 == 0 and both images 16-byte aligned -- the staging then reads
// aligned float4 groups (columns TX - 12 .. TX + 43, the outer two on each side
// dropped).
__global__ void __launch_bounds__(kSsimThreads) k_ssim(const float* __restrict__ x, const float* __restrict__ y,
                                                       const int* __restrict__ meas_sel, int H, int W, int tiles_x,
                                                       int tiles_per_view, int n_tiles, const Win win,
                                                       float l1_scale, float ssim_scale, float* __restrict__ grad,
                                                       float* __restrict__ partials, unsigned int* __restrict__ arrive,
                                                       float lam, float inv_n, int vec4, float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SsimSmem& S = *reinterpret_cast<SsimSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int v = tile / tiles_per_view, lt = tile - v * tiles_per_view;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int TY = ty * kT, TX = tx * kT;
    const float* xv = x + (size_t)v * H * W;
    const float* yv = y + (size_t)(meas_sel ? meas_sel[v] : v) * H * W;
    pdl_trigger();
    // the measurement first (no earlier kernel writes it), then, once the kernel
    // that renders x has finished, the render
    stage_tile(S.sy, yv, TY, TX, H, W, tid, vec4);
    pdl_wait();
    stage_tile(S.sx, xv, TY, TX, H, W, tid, vec4);
    __syncthreads();
    // The moments are taken of x - cs and y - cs (cs: the mean of both images at the
    // staged region's centre; pixels outside the image, x = y = 0, become -cs), so that
    // the (co)variances E[x'y'] - mu_x' mu_y' do not cancel the squared means of
    // bright, smooth regions; they equal those of x and y because the window sums to
    // one.  mu_x = mu_x' + cs enters the luminance term.
    const float cs = 0.5f * (S.sx[kS / 2][kS / 2] + S.sy[kS / 2][kS / 2]);
    // Each pass is register-blocked along its filter direction: a thread computes a
    // run of outputs from one sliding set of inputs (every input loaded once), and
    // the lanes of a warp take consecutive rows (horizontal passes) or columns
    // (vertical passes), so shared-memory accesses are free of bank conflicts.
    // Horizontal pass of x, y, xx, yy, xy: rows 0..kS-1, output columns 0..kM-1.
    {
        constexpr int RB = 6, NSEG = kM / RB;  // 7 runs of 6 columns per row
        static_assert(kM % RB == 0 && NSEG * kS <= kSsimThreads, "one pass");
        if (tid < NSEG * kS) {
            const int r = tid % kS, c0 = (tid / kS) * RB;
            float acc[RB][5];
#pragma unroll
            for (int o = 0; o < RB; ++o)
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[o][q] = 0.f;
#pragma unroll
            for (int i = 0; i < RB + 10; ++i) {
                const float xa = S.sx[r][c0 + i] - cs, ya = S.sy[r][c0 + i] - cs;
                const float f[5] = {xa, ya, xa * xa, ya * ya, xa * ya};
#pragma unroll
                for (int o = 0; o < RB; ++o) {
                    const int j = i - o;
                    if (j >= 0 && j <= 10) {
#pragma unroll
                        for (int q = 0; q < 5; ++q) acc[o][q] = fmaf(win.w[j], f[q], acc[o][q]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < RB; ++o)
#pragma unroll
                for (int q = 0; q < 5; ++q) S.u.h[q][r][c0 + o] = acc[o][q];
        }
    }
    __syncthreads();
    // Vertical pass -> moments, SSIM term and its derivatives on the tile plus halo.
    float sS = 0.f, sL1 = 0.f;
    {
        constexpr int RB = 4, NSEG = (kM + RB - 1) / RB;  // 11 runs of (up to) 4 rows per column
        static_assert(NSEG * kM <= kSsimThreads, "one pass");
        if (tid < NSEG * kM) {
            const int c = tid % kM, r0 = (tid / kM) * RB;
            float m[RB][5];
#pragma unroll
            for (int o = 0; o < RB; ++o)
#pragma unroll
                for (int q = 0; q < 5; ++q) m[o][q] = 0.f;
#pragma unroll
            for (int i = 0; i < RB + 10; ++i) {
                if (r0 + i < kS) {
                    float hq[5];
#pragma unroll
                    for (int q = 0; q < 5; ++q) hq[q] = S.u.h[q][r0 + i][c];
#pragma unroll
                    for (int o = 0; o < RB; ++o) {
                        const int j = i - o;
                        if (j >= 0 && j <= 10) {
#pragma unroll
                            for (int q = 0; q < 5; ++q) m[o][q] = fmaf(win.w[j], hq[q], m[o][q]);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                const int r = r0 + o;
                if (r >= kM) break;
                const int gy = TY - kR + r, gx = TX - kR + c;
                float dm = 0.f, dxx = 0.f, dxy = 0.f;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const float mxs = m[o][0], mys = m[o][1];       // means of the shifted images
                    const float mx = mxs + cs, my = mys + cs;
                    const float sxx = m[o][2] - mxs * mxs, syy = m[o][3] - mys * mys, sxy = m[o][4] - mxs * mys;
                    const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
                    const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
                    const float iB = __frcp_rn(B1 * B2);
                    const float Sv = A1 * A2 * iB;
                    // dS/dmu_x' with E_x'x', E_x'y' held: A1, B1 move with mu_x = mu_x' + cs,
                    // A2, B2 with -mu_x'^2 and -mu_x' mu_y'
                    dm = (2.f * (my * A2 - mys * A1) - 2.f * Sv * (mx * B2 - mxs * B1)) * iB;
                    dxx = -Sv * (B1 * iB);                   // -S / B2
                    dxy = 2.f * A1 * iB;
                    if (r >= kR && r < kR + kT && c >= kR && c < kR + kT) {  // this tile's own pixels
                        sS += 1.f - Sv;
                        sL1 += fabsf(S.sx[r + kR][c + kR] - S.sy[r + kR][c + kR]);
                    }
                }
                S.d[0][r][c] = dm;
                S.d[1][r][c] = dxx;
                S.d[2][r][c] = dxy;
            }
        }
    }
    __syncthreads();
    // Horizontal pass of the derivative maps: rows 0..kM-1, output columns 0..kT-1.
    {
        constexpr int RB = 8, NSEG = kT / RB;  // 4 runs of 8 columns per row
        static_assert(kT % RB == 0 && NSEG * kM <= kSsimThreads, "one pass");
        if (tid < NSEG * kM) {
            const int r = tid % kM, c0 = (tid / kM) * RB;
            float acc[RB][3];
#pragma unroll
            for (int o = 0; o < RB; ++o)
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[o][q] = 0.f;
#pragma unroll
            for (int i = 0; i < RB + 10; ++i) {
                const float f[3] = {S.d[0][r][c0 + i], S.d[1][r][c0 + i], S.d[2][r][c0 + i]};
#pragma unroll
                for (int o = 0; o < RB; ++o) {
                    const int j = i - o;
                    if (j >= 0 && j <= 10) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) acc[o][q] = fmaf(win.w[j], f[q], acc[o][q]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < RB; ++o)
#pragma unroll
                for (int q = 0; q < 3; ++q) S.u.g[q][r][c0 + o] = acc[o][q];
        }
    }
    __syncthreads();
    // Vertical pass -> d loss / d render on the tile's own pixels.
    {
        constexpr int RB = 4, NSEG = kT / RB;  // 8 runs of 4 rows per column
        static_assert(kT % RB == 0 && NSEG * kT <= kSsimThreads, "one pass");
        if (tid < NSEG * kT) {
            const int c = tid % kT, r0 = (tid / kT) * RB;
            float b[RB][3];
#pragma unroll
            for (int o = 0; o < RB; ++o)
#pragma unroll
                for (int q = 0; q < 3; ++q) b[o][q] = 0.f;
#pragma unroll
            for (int i = 0; i < RB + 10; ++i) {
                const float f[3] = {S.u.g[0][r0 + i][c], S.u.g[1][r0 + i][c], S.u.g[2][r0 + i][c]};
#pragma unroll
                for (int o = 0; o < RB; ++o) {
                    const int j = i - o;
                    if (j >= 0 && j <= 10) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) b[o][q] = fmaf(win.w[j], f[q], b[o][q]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                const int r = r0 + o;
                const int gy = TY + r, gx = TX + c;
                if (gy >= H || gx >= W) continue;
                const float xp = S.sx[r + 2 * kR][c + 2 * kR], yp = S.sy[r + 2 * kR][c + 2 * kR];
                const float dd = xp - yp;
                const float sgn = (dd > 0.f) ? 1.f : ((dd < 0.f) ? -1.f : 0.f);
                grad[((size_t)v * H + gy) * W + gx] =
                    l1_scale * sgn - ssim_scale * (b[o][0] + 2.f * (xp - cs) * b[o][1] + (yp - cs) * b[o][2]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sS += __shfl_xor_sync(0xffffffffu, sS, o);
        sL1 += __shfl_xor_sync(0xffffffffu, sL1, o);
    }
    if ((tid & 31) == 0) {
        S.red[0][tid >> 5] = sS;
        S.red[1][tid >> 5] = sL1;
    }
    __syncthreads();
    if (tid == kArriveThread) {
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int w = 0; w < kSsimThreads / 32; ++w) {
            a += S.red[0][w];
            b += S.red[1][w];
        }
        partials[2 * tile] = a;
        partials[2 * tile + 1] = b;
        __threadfence();
        S.last = atomicAdd(arrive, 1u) == (unsigned)(n_tiles - 1);
    }
    __syncthreads();
    if (!S.last) return;
    __threadfence();
    // the tiles' partials in a fixed order: a strided sum per thread, then warp and CTA trees
    float a = 0.f, b = 0.f;
    for (int k = tid; k < n_tiles; k += kSsimThreads) {
        a += __ldcg(partials + 2 * k);
        b += __ldcg(partials + 2 * k + 1);
    }
    __syncthreads();  // S.red is reused
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0) {
        S.red[0][tid >> 5] = a;
        S.red[1][tid >> 5] = b;
    }
    __syncthreads();
    if (tid == 0) {
        float sa = 0.f, sb = 0.f;
#pragma unroll
        for (int w = 0; w < kSsimThreads / 32; ++w) {
            sa += S.red[0][w];
            sb += S.red[1][w];
        }
        *loss = inv_n * sb + lam * (inv_n * sa);
    }
}

// loss = a0 * sum(p[2k+1]) + a1 * (1 - b1 * sum(p[2k]))  (projection loss), or
// loss = a0 * sum(p[k]) for a stride-1 list (TV): mode selects.
__global__ void __launch_bounds__(256) k_finalize(const float* __restrict__ p, int n, int mode, float a0, float a1,
                                                  float b1, float* __restrict__ loss) {
    __shared__ double red[2][256];
    double s0 = 0.0, s1 = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) {
        if (mode == 0) {
            s0 += p[2 * k];
            s1 += p[2 * k + 1];
        } else {
            s1 += p[k];
        }
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (mode == 0)
            *loss = (float)(a0 * red[1][0] + a1 * (1.0 - b1 * red[0][0]));
        else
            *loss = (float)(a0 * red[1][0]);
    }
}

__global__ void __launch_bounds__(256) k_tv3d(const float* __restrict__ vol, int D, long long n, float inv_cnt,
                                              float lam, float* __restrict__ grad, float* __restrict__ partials) {
    __shared__ float red[8];
    const float s = tv3d_block(vol, D, n, inv_cnt, lam, grad, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// The TV loss: lam inv_cnt x the fixed-order sum of the per-block partials.
__global__ void __launch_bounds__(256) k_tv_sum(const float* __restrict__ p, int n, float scale,
                                                float* __restrict__ loss) {
    __shared__ double red[256];
    const double s = sum_partials_256(p, n, red);
    if (threadIdx.x == 0) *loss = (float)(scale * s);
}

// Isotropic TV: n(x) = sqrt(sum_k d_k(x)^2 + eps) with d_k(x) = V(x + e_k) - V(x)
// (0 on the far face).  V(x) enters its own n with d(n)/dV(x) = -sum_k d_k(x) / n(x)
// and the n of each backward neighbour x - e_k with d_k(x - e_k) / n(x - e_k), so a
// thread reads its voxel, its 3 forward and 3 backward neighbours and the 6
// diagonal ones that the backward neighbours' differences need (L1-resident).
__device__ __forceinline__ float tv_fwd_diff(const float* vg, long long l, long long st, int co, int D, float c) {
    return (co + 1 < D) ? vg[l + st] - c : 0.f;
}

__global__ void __launch_bounds__(256) k_tv3d_iso(const float* __restrict__ vol, int D, long long n, float inv_cnt,
                                                  float lam, float eps, float* __restrict__ grad,
                                                  float* __restrict__ partials) {
    __shared__ float red[8];
    const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
    float part = 0.f;
    if (idx < n) {
        const long long D3 = (long long)D * D * D;
        const long long g = idx / D3;
        const long long l = idx - g * D3;
        const int z = (int)(l / ((long long)D * D)), y = (int)((l / D) % D), x = (int)(l % D);
        const float* vg = vol + g * D3;
        const float c = vg[l];
        const long long st[3] = {1, D, (long long)D * D};
        const int co[3] = {x, y, z};
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = tv_fwd_diff(vg, l, st[a], co[a], D, c);
        const float nrm = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps);
        part = nrm;
        float gr = -(d[0] + d[1] + d[2]) / nrm;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (co[a] == 0) continue;
            const long long lb = l - st[a];
            const float cb = vg[lb];
            const float da = c - cb;
            float s = da * da + eps;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                const float db = tv_fwd_diff(vg, lb, st[b], co[b], D, cb);
                s += db * db;
            }
            gr += da / sqrtf(s);
        }
        grad[idx] = lam * inv_cnt * gr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

Win gaussian_window() {
    double g[11], s = 0;
    for (int k = 0; k < 11; ++k) {
        const double d = k - 5.0;
        g[k] = exp(-d * d / (2 * 1.5 * 1.5));
        s += g[k];
    }
    Win w;
    for (int k = 0; k < 11; ++k) w.w[k] = (float)(g[k] / s);
    return w;
}

struct LossLayout {
    size_t partials, arrive, fixed;
    int tiles_x, tiles_y;
    long long n_tiles;
};

LossLayout loss_layout(int V, int H, int W) {
    LossLayout L;
    L.tiles_x = (W + kT - 1) / kT;
    L.tiles_y = (H + kT - 1) / kT;
    L.n_tiles = (long long)V * L.tiles_x * L.tiles_y;
    Layout lay;
    L.partials = lay.take(8 * (size_t)L.n_tiles);
    L.arrive = lay.take(sizeof(unsigned int));
    L.fixed = lay.off;
    return L;
}

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API size_t r2g_loss_workspace_size(int32_t V, int32_t H, int32_t W) {
    if (V < 1 || H < 1 || W < 1) return 0;
    return loss_layout(V, H, W).fixed;
}

r2g_status r2g::projection_loss_clear(int32_t V, int32_t H, int32_t W, void* ws, size_t ws_bytes,
                                      cudaStream_t stream) {
    if (V < 1 || H < 1 || W < 1 || !ws) return fail(R2G_E_INVAL, "bad loss workspace");
    const LossLayout L = loss_layout(V, H, W);
    if (ws_bytes < L.fixed) return fail(R2G_E_INVAL, "loss workspace needs %zu bytes", L.fixed);
    if (cudaMemsetAsync(static_cast<char*>(ws) + L.arrive, 0, sizeof(unsigned int), stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "clearing the loss arrival counter: %s", cudaGetErrorString(cudaGetLastError()));
    return R2G_OK;
}

r2g_status r2g::projection_loss_impl(int32_t V, int32_t H, int32_t W, const float* render, const float* meas,
                                     const int* meas_sel, float lambda_ssim, float* loss, float* drender, void* ws,
                                     size_t ws_bytes, cudaStream_t stream, bool clear_arrival) {
    if (V < 1 || H < 1 || W < 1 || H > 32768 || W > 32768) return fail(R2G_E_INVAL, "bad image shape");
    if (!render || !meas || !loss || !drender || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    const LossLayout L = loss_layout(V, H, W);
    if (ws_bytes < L.fixed) return fail(R2G_E_INVAL, "loss workspace needs %zu bytes", L.fixed);
    if (L.n_tiles >= (1ll << 31)) return fail(R2G_E_INVAL, "image too large");
    const Win win = gaussian_window();
    char* base = static_cast<char*>(ws);
    float* partials = reinterpret_cast<float*>(base + L.partials);
    unsigned int* arrive = reinterpret_cast<unsigned int*>(base + L.arrive);
    // the kernel's shared memory exceeds the 48 KB default: opt in once per device
    // (idempotent, so racing first calls are harmless)
    static bool smem_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !smem_set[dev]) {
        if (cudaFuncSetAttribute(k_ssim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SsimSmem)) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_ssim, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return fail(R2G_E_CUDA, "r2g_projection_loss: shared memory attribute (%s)",
                        cudaGetErrorString(cudaGetLastError()));
        if (dev >= 0 && dev < 64) smem_set[dev] = true;
    }
    const int tpv = L.tiles_x * L.tiles_y;
    const double N = (double)V * H * W;
    const int vec4 = (W % 4 == 0) && reinterpret_cast<uintptr_t>(render) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(meas) % 16 == 0;
    prof_begin(P_LOSS, stream);
    if (clear_arrival) cudaMemsetAsync(arrive, 0, sizeof(unsigned int), stream);
    launch_pdl(k_ssim, dim3((unsigned)L.n_tiles), dim3(kSsimThreads), sizeof(SsimSmem), stream, render, meas, meas_sel,
               H, W, L.tiles_x, tpv, (int)L.n_tiles, win, (float)(1.0 / N), (float)(lambda_ssim / N), drender,
               partials, arrive, lambda_ssim, (float)(1.0 / N), vec4, loss);
    prof_end(P_LOSS, stream);
    note_launches(1);
    return check_launch("r2g_projection_loss");
}

R2G_API r2g_status r2g_projection_loss(int32_t V, int32_t H, int32_t W, const float* render, const float* meas,
                                       float lambda_ssim, float* loss, float* drender, void* ws, size_t ws_bytes,
                                       r2g_stream stream) {
    return projection_loss_impl(V, H, W, render, meas, nullptr, lambda_ssim, loss, drender, ws, ws_bytes, stream);
}

R2G_API size_t r2g_tv_workspace_size(int32_t G, int32_t D) {
    if (G < 1 || D < 2 || D > 1024) return 0;
    const long long n = (long long)G * D * D * D;
    return align_up(4 * (size_t)((n + 255) / 256));
}

R2G_API r2g_status r2g_tv3d(int32_t G, int32_t D, const float* vol, float lambda_tv, float* loss, float* dvol,
                            void* ws, size_t ws_bytes, r2g_stream stream) {
    if (G < 1 || D < 2 || D > 1024) return fail(R2G_E_INVAL, "bad TV volume shape G=%d D=%d", G, D);
    if (!vol || !loss || !dvol || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    const long long n = (long long)G * D * D * D;
    const long long blocks = (n + 255) / 256;
    if (blocks >= (1ll << 31)) return fail(R2G_E_INVAL, "TV volume too large");
    if (ws_bytes < 4 * (size_t)blocks) return fail(R2G_E_INVAL, "TV workspace needs %zu bytes", 4 * (size_t)blocks);
    float* partials = static_cast<float*>(ws);
    // every axis has D^2 (D - 1) forward differences
    const float inv_cnt = (float)(1.0 / ((double)D * D * (D - 1)));
    prof_begin(P_TV, stream);
    k_tv3d<<<(unsigned)blocks, 256, 0, stream>>>(vol, D, n, inv_cnt, lambda_tv, dvol, partials);
    k_tv_sum<<<1, 256, 0, stream>>>(partials, (int)blocks, lambda_tv * inv_cnt, loss);
    prof_end(P_TV, stream);
    note_launches(2);
    return check_launch("r2g_tv3d");
}

R2G_API r2g_status r2g_tv3d_iso(int32_t G, int32_t D, const float* vol, float lambda_tv, float eps, float* loss,
                                float* dvol, void* ws, size_t ws_bytes, r2g_stream stream) {
    if (G < 1 || D < 2 || D > 1024) return fail(R2G_E_INVAL, "bad TV volume shape G=%d D=%d", G, D);
    if (!vol || !loss || !dvol || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (!(eps > 0.f)) return fail(R2G_E_INVAL, "r2g_tv3d_iso: eps must be > 0 (got %g)", (double)eps);
    const long long n = (long long)G * D * D * D;
    const long long blocks = (n + 255) / 256;
    if (blocks >= (1ll << 31)) return fail(R2G_E_INVAL, "TV volume too large");
    if (ws_bytes < 4 * (size_t)blocks) return fail(R2G_E_INVAL, "TV workspace needs %zu bytes", 4 * (size_t)blocks);
    float* partials = static_cast<float*>(ws);
    // the mean over the D^3 voxels of each volume
    const float inv_cnt = (float)(1.0 / ((double)D * D * D));
    prof_begin(P_TV, stream);
    k_tv3d_iso<<<(unsigned)blocks, 256, 0, stream>>>(vol, D, n, inv_cnt, lambda_tv, eps, dvol, partials);
    k_finalize<<<1, 256, 0, stream>>>(partials, (int)blocks, 1, lambda_tv * inv_cnt, 0.f, 0.f, loss);
    prof_end(P_TV, stream);
    note_launches(2);
    return check_launch("r2g_tv3d_iso");
}
