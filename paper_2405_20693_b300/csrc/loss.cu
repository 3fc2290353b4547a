// loss.cu -- the training losses of Eq. 8 on sm_103a, forward and gradient fused.
//
// Projection loss L1 + lambda_ssim (1 - SSIM) over [V][H][W]:
//   k_ssim_maps   one CTA per 32x32 output tile of one view: the tile plus a
//                 5-pixel halo of render x and measurement y is staged in shared
//                 memory (zeros outside the image), the 11-tap Gaussian window is
//                 applied separably to x, y, xx, yy, xy, and each pixel's SSIM
//                 term S and its partial derivatives with respect to the local
//                 moments (dS/dmu_x, dS/dE_xx, dS/dE_xy) are formed.  Writes the
//                 three derivative maps and per-CTA partial sums of S and |x - y|.
//   k_ssim_grad   one CTA per tile again: the derivative maps plus halo are
//                 filtered with the same window (the adjoint of a zero-padded
//                 symmetric filter is itself) and combined with x, y and the L1
//                 sign into d loss / d render.
//                 Its block 0 also sums the per-tile partials of k_ssim_maps in a
//                 fixed order into the loss (deterministic).
//   k_finalize    (TV) one CTA sums the per-CTA partials in a fixed order.
// 3D TV: k_tv3d forms each voxel's gradient from its six neighbours and a CTA
// partial of the loss; k_finalize sums the partials.
#include <math.h>

#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr int kT = 32;            // output tile edge
constexpr int kR = 5;             // window radius
constexpr int kE = kT + 2 * kR;   // staged edge

// Normalised 1D Gaussian window (sigma 1.5), passed by value to each launch.
struct Win {
    float w[11];
};

constexpr float kC1 = 1e-4f;      // (0.01 L)^2, L = 1
constexpr float kC2 = 9e-4f;      // (0.03 L)^2

// meas_sel (optional, device): view v of the batch is compared with measurement
// meas_sel[v] of y.
__global__ void __launch_bounds__(256) k_ssim_maps(const float* __restrict__ x, const float* __restrict__ y,
                                                   const int* __restrict__ meas_sel, int H,
                                                   int W, int tiles_x, int tiles_per_view, const Win win,
                                                   float* __restrict__ dmu,
                                                   float* __restrict__ dxx, float* __restrict__ dxy,
                                                   float* __restrict__ partials) {
    __shared__ float sx[kE][kE + 1], sy[kE][kE + 1];
    __shared__ float h[5][kE][kT + 1];
    __shared__ float red[2][8];
    const int tile = blockIdx.x;
    const int v = tile / tiles_per_view, lt = tile - v * tiles_per_view;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int Y0 = ty * kT - kR, X0 = tx * kT - kR;
    const float* xv = x + (size_t)v * H * W;
    const float* yv = y + (size_t)(meas_sel ? meas_sel[v] : v) * H * W;
    for (int k = threadIdx.x; k < kE * kE; k += 256) {
        const int r = k / kE, c = k - r * kE;
        const int gy = Y0 + r, gx = X0 + c;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        sx[r][c] = in ? xv[(size_t)gy * W + gx] : 0.f;
        sy[r][c] = in ? yv[(size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    // horizontal pass: rows 0..kE-1, output columns 0..kT-1
    for (int k = threadIdx.x; k < kE * kT; k += 256) {
        const int r = k / kT, c = k - r * kT;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
        for (int j = 0; j < 11; ++j) {
            const float w = win.w[j];
            const float xa = sx[r][c + j], ya = sy[r][c + j];
            a0 = fmaf(w, xa, a0);
            a1 = fmaf(w, ya, a1);
            a2 = fmaf(w, xa * xa, a2);
            a3 = fmaf(w, ya * ya, a3);
            a4 = fmaf(w, xa * ya, a4);
        }
        h[0][r][c] = a0;
        h[1][r][c] = a1;
        h[2][r][c] = a2;
        h[3][r][c] = a3;
        h[4][r][c] = a4;
    }
    __syncthreads();
    float sS = 0.f, sL1 = 0.f;
    for (int k = threadIdx.x; k < kT * kT; k += 256) {
        const int r = k / kT, c = k - r * kT;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 11; ++j) {
            const float w = win.w[j];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmaf(w, h[q][r + j][c], m[q]);
        }
        const int gy = ty * kT + r, gx = tx * kT + c;
        if (gy < H && gx < W) {
            const float mx = m[0], my = m[1];
            const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
            const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
            const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
            const float iB = 1.f / (B1 * B2);
            const float S = A1 * A2 * iB;
            const size_t o = ((size_t)v * H + gy) * W + gx;
            dmu[o] = (2.f * my * (A2 - A1) - 2.f * mx * S * (B2 - B1)) * iB;
            dxx[o] = -S / B2;
            dxy[o] = 2.f * A1 * iB;
            sS += S;
            sL1 += fabsf(sx[r + kR][c + kR] - sy[r + kR][c + kR]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sS += __shfl_xor_sync(0xffffffffu, sS, o);
        sL1 += __shfl_xor_sync(0xffffffffu, sL1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sS;
        red[1][threadIdx.x >> 5] = sL1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < 8; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        partials[2 * tile] = a;
        partials[2 * tile + 1] = b;
    }
}

__global__ void __launch_bounds__(256) k_ssim_grad(const float* __restrict__ x, const float* __restrict__ y,
                                                   const int* __restrict__ meas_sel, int H,
                                                   int W, int tiles_x, int tiles_per_view, const Win win,
                                                   const float* __restrict__ dmu, const float* __restrict__ dxx,
                                                   const float* __restrict__ dxy, float l1_scale, float ssim_scale,
                                                   float* __restrict__ grad, const float* __restrict__ partials,
                                                   int n_tiles, float lam, double inv_n, float* __restrict__ loss) {
    __shared__ float s[3][kE][kE + 1];
    __shared__ float h[3][kE][kT + 1];
    __shared__ double red[2][256];
    const int tile = blockIdx.x;
    const int v = tile / tiles_per_view, lt = tile - v * tiles_per_view;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int Y0 = ty * kT - kR, X0 = tx * kT - kR;
    const size_t vb = (size_t)v * H * W;
    for (int k = threadIdx.x; k < kE * kE; k += 256) {
        const int r = k / kE, c = k - r * kE;
        const int gy = Y0 + r, gx = X0 + c;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const size_t o = vb + (size_t)gy * W + gx;
        s[0][r][c] = in ? dmu[o] : 0.f;
        s[1][r][c] = in ? dxx[o] : 0.f;
        s[2][r][c] = in ? dxy[o] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kE * kT; k += 256) {
        const int r = k / kT, c = k - r * kT;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int j = 0; j < 11; ++j) {
            const float w = win.w[j];
            a0 = fmaf(w, s[0][r][c + j], a0);
            a1 = fmaf(w, s[1][r][c + j], a1);
            a2 = fmaf(w, s[2][r][c + j], a2);
        }
        h[0][r][c] = a0;
        h[1][r][c] = a1;
        h[2][r][c] = a2;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kT * kT; k += 256) {
        const int r = k / kT, c = k - r * kT;
        const int gy = ty * kT + r, gx = tx * kT + c;
        if (gy >= H || gx >= W) continue;
        float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
        for (int j = 0; j < 11; ++j) {
            const float w = win.w[j];
            b0 = fmaf(w, h[0][r + j][c], b0);
            b1 = fmaf(w, h[1][r + j][c], b1);
            b2 = fmaf(w, h[2][r + j][c], b2);
        }
        const size_t o = vb + (size_t)gy * W + gx;
        const float xv = x[o], yv = y[(size_t)(meas_sel ? meas_sel[v] : v) * H * W + (size_t)gy * W + gx];
        const float d = xv - yv;
        const float sgn = (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f);
        grad[o] = l1_scale * sgn - ssim_scale * (b0 + 2.f * xv * b1 + yv * b2);
    }
    // The per-tile partial sums come from the previous kernel, so any one block can
    // form the loss: block 0 sums them in a fixed order.
    if (blockIdx.x == 0) {
        double sS = 0.0, sL1 = 0.0;
        for (int k = threadIdx.x; k < n_tiles; k += 256) {
            sS += partials[2 * k];
            sL1 += partials[2 * k + 1];
        }
        red[0][threadIdx.x] = sS;
        red[1][threadIdx.x] = sL1;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                red[0][threadIdx.x] += red[0][threadIdx.x + o];
                red[1][threadIdx.x] += red[1][threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) *loss = (float)(inv_n * red[1][0] + lam * (1.0 - inv_n * red[0][0]));
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
    size_t dmu, dxx, dxy, partials, fixed;
    int tiles_x, tiles_y;
    long long n_tiles;
};

LossLayout loss_layout(int V, int H, int W) {
    LossLayout L;
    L.tiles_x = (W + kT - 1) / kT;
    L.tiles_y = (H + kT - 1) / kT;
    L.n_tiles = (long long)V * L.tiles_x * L.tiles_y;
    const size_t n = (size_t)V * H * W;
    Layout lay;
    L.dmu = lay.take(4 * n);
    L.dxx = lay.take(4 * n);
    L.dxy = lay.take(4 * n);
    L.partials = lay.take(8 * (size_t)L.n_tiles);
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

r2g_status r2g::projection_loss_impl(int32_t V, int32_t H, int32_t W, const float* render, const float* meas,
                                     const int* meas_sel, float lambda_ssim, float* loss, float* drender, void* ws,
                                     size_t ws_bytes, cudaStream_t stream) {
    if (V < 1 || H < 1 || W < 1 || H > 32768 || W > 32768) return fail(R2G_E_INVAL, "bad image shape");
    if (!render || !meas || !loss || !drender || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    const LossLayout L = loss_layout(V, H, W);
    if (ws_bytes < L.fixed) return fail(R2G_E_INVAL, "loss workspace needs %zu bytes", L.fixed);
    if (L.n_tiles >= (1ll << 31)) return fail(R2G_E_INVAL, "image too large");
    const Win win = gaussian_window();
    char* base = static_cast<char*>(ws);
    float* dmu = reinterpret_cast<float*>(base + L.dmu);
    float* dxx = reinterpret_cast<float*>(base + L.dxx);
    float* dxy = reinterpret_cast<float*>(base + L.dxy);
    float* partials = reinterpret_cast<float*>(base + L.partials);
    const int tpv = L.tiles_x * L.tiles_y;
    prof_begin(P_LOSS, stream);
    k_ssim_maps<<<(unsigned)L.n_tiles, 256, 0, stream>>>(render, meas, meas_sel, H, W, L.tiles_x, tpv, win, dmu,
                                                          dxx, dxy, partials);
    const double N = (double)V * H * W;
    k_ssim_grad<<<(unsigned)L.n_tiles, 256, 0, stream>>>(render, meas, meas_sel, H, W, L.tiles_x, tpv, win, dmu,
                                                          dxx, dxy,
                                                          (float)(1.0 / N), (float)(lambda_ssim / N), drender,
                                                          partials, (int)L.n_tiles, lambda_ssim, 1.0 / N, loss);
    prof_end(P_LOSS, stream);
    note_launches(2);
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
    k_finalize<<<1, 256, 0, stream>>>(partials, (int)blocks, 1, lambda_tv * inv_cnt, 0.f, 0.f, loss);
    prof_end(P_TV, stream);
    note_launches(2);
    return check_launch("r2g_tv3d");
}
