// metrics.cu -- the reconstruction metrics of Sec. 5.1 on the GPU: PSNR over the
// whole volume and SSIM averaged over the 2D slices of the three orientations.
//
// For a [Z][Y][X] volume (z the rotation axis) the axial slices are the z = const
// images (rows y, columns x), the coronal ones y = const (rows z, columns x) and
// the sagittal ones x = const (rows z, columns y).  Slice SSIM is Wang et al.'s
// with an 11 x 11 Gaussian window (sigma 1.5), zero-padded "same" filtering,
// C1 = (0.01 L)^2, C2 = (0.03 L)^2 and L = 1, averaged over the slice's pixels;
// each orientation's value is the mean over its slices, and the 3D SSIM the mean
// of the three.  PSNR = 10 log10(1 / MSE).
//
//   k_transpose_zyx  copies of both volumes in [x][z][y] order, so that sagittal
//                 slices are read like the others (rows contiguous);
//   k_slice_ssim  one CTA (128 threads) per 32 x 32 output tile of one slice of
//                 one orientation: both volumes' tiles staged with a 5-voxel halo
//                 (zeros outside the slice), the window applied separably to a, b,
//                 a^2, b^2, ab with register-blocked runs (4 columns, 8 rows per
//                 thread), the SSIM term summed over the tile's in-slice pixels
//                 (double) into a per-tile partial;
//   k_sq_err      per-CTA partial sums of (a - b)^2 (double), grid-stride;
//   k_metrics_fin one CTA sums the partials in a fixed order (deterministic).
#include <math.h>

#include "r2g_internal.cuh"

namespace r2g {
namespace {

constexpr int kMT = 32;              // output tile edge
constexpr int kMR = 5;               // window radius
constexpr int kMS = kMT + 2 * kMR;   // staged edge
constexpr int kMetThreads = 128;
constexpr int kSqBlocks = 148 * 4;
constexpr float kMC1 = 1e-4f, kMC2 = 9e-4f;

struct MWin {
    float w[11];
};

struct Orient {
    long long ss, sr, sc;  // element strides of slice, row, column
    int n, H, W;           // slices, rows, columns
    int tiles_x, tiles;    // tiles per row of tiles, tiles per slice
    long long first;       // first CTA of this orientation
};

struct Orients {
    Orient o[3];
};

// Register-blocked separable window: the horizontal pass gives each thread a run of
// kMHR output columns of one staged row (the 14 inputs loaded once, their three
// products formed once), the vertical pass a run of kMVR output rows of one column
// (each of the 18 staged rows of the five moments loaded once).  Each output still
// accumulates its taps in window order, k = 0 .. 10, so the filtered moments are
// those of the tap-by-tap loop.
constexpr int kMHR = 4;  // output columns per thread, horizontal pass
constexpr int kMVR = 8;  // output rows per thread, vertical pass
static_assert(kMetThreads == kMT * (kMT / kMVR), "one vertical run per thread");

__global__ void __launch_bounds__(kMetThreads) k_slice_ssim(const float* __restrict__ a, const float* __restrict__ b,
                                                            const float* __restrict__ ta,
                                                            const float* __restrict__ tb, Orients os, MWin win,
                                                            double* __restrict__ partials) {
    __shared__ float sa[kMS][kMS + 1], sb[kMS][kMS + 1];
    __shared__ float h[5][kMS][kMT + 1];
    __shared__ double red[kMetThreads / 32];
    const long long cta = blockIdx.x;
    const int oi = cta >= os.o[2].first ? 2 : (cta >= os.o[1].first ? 1 : 0);
    const Orient o = os.o[oi];
    const long long local = cta - o.first;
    const int s = (int)(local / o.tiles);
    const int tile = (int)(local - (long long)s * o.tiles);
    const int r0 = (tile / o.tiles_x) * kMT, c0 = (tile % o.tiles_x) * kMT;
    const float* pa = (oi == 2 ? ta : a) + (long long)s * o.ss;
    const float* pb = (oi == 2 ? tb : b) + (long long)s * o.ss;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // staging: a warp per row (rows warp, warp + 4, ...), the lanes along it (two
    // passes cover the 42 columns), all of a thread's loads issued before its stores
    {
        const int gc0 = c0 - kMR + lane, gc1 = gc0 + 32;
        const bool in0 = gc0 >= 0 && gc0 < o.W, in1 = lane < kMS - 32 && gc1 >= 0 && gc1 < o.W;
#pragma unroll 2
        for (int r = warp; r < kMS; r += kMetThreads / 32) {
            const int gr = r0 + r - kMR;
            const bool rin = gr >= 0 && gr < o.H;
            const long long ro = (long long)gr * o.sr;
            const float va0 = rin && in0 ? pa[ro + (long long)gc0 * o.sc] : 0.f;
            const float vb0 = rin && in0 ? pb[ro + (long long)gc0 * o.sc] : 0.f;
            const float va1 = rin && in1 ? pa[ro + (long long)gc1 * o.sc] : 0.f;
            const float vb1 = rin && in1 ? pb[ro + (long long)gc1 * o.sc] : 0.f;
            sa[r][lane] = va0;
            sb[r][lane] = vb0;
            if (lane < kMS - 32) {
                sa[r][lane + 32] = va1;
                sb[r][lane + 32] = vb1;
            }
        }
    }
    __syncthreads();
    // horizontal pass: h[m][r][c] = sum_k w_k P_m(r, c + k), c over the 32 output columns
    for (int item = tid; item < kMS * (kMT / kMHR); item += kMetThreads) {
        const int r = item / (kMT / kMHR), cb = (item - r * (kMT / kMHR)) * kMHR;
        float m0[kMHR], m1[kMHR], m2[kMHR], m3[kMHR], m4[kMHR];
#pragma unroll
        for (int i = 0; i < kMHR; ++i) m0[i] = m1[i] = m2[i] = m3[i] = m4[i] = 0.f;
#pragma unroll
        for (int j = 0; j < kMHR + 10; ++j) {
            const float x = sa[r][cb + j], y = sb[r][cb + j];
            const float xx = x * x, yy = y * y, xy = x * y;
#pragma unroll
            for (int i = 0; i < kMHR; ++i) {
                const int k = j - i;  // tap of input j for output i (compile time)
                if (k >= 0 && k <= 10) {
                    const float w = win.w[k];
                    m0[i] = fmaf(w, x, m0[i]);
                    m1[i] = fmaf(w, y, m1[i]);
                    m2[i] = fmaf(w, xx, m2[i]);
                    m3[i] = fmaf(w, yy, m3[i]);
                    m4[i] = fmaf(w, xy, m4[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kMHR; ++i) {
            h[0][r][cb + i] = m0[i];
            h[1][r][cb + i] = m1[i];
            h[2][r][cb + i] = m2[i];
            h[3][r][cb + i] = m3[i];
            h[4][r][cb + i] = m4[i];
        }
    }
    __syncthreads();
    // vertical pass: column c, output rows rb .. rb + kMVR - 1
    const int c = tid % kMT, rb = (tid / kMT) * kMVR;
    float mx[kMVR], my[kMVR], exx[kMVR], eyy[kMVR], exy[kMVR];
#pragma unroll
    for (int i = 0; i < kMVR; ++i) mx[i] = my[i] = exx[i] = eyy[i] = exy[i] = 0.f;
#pragma unroll
    for (int j = 0; j < kMVR + 10; ++j) {
        const float v0 = h[0][rb + j][c], v1 = h[1][rb + j][c], v2 = h[2][rb + j][c], v3 = h[3][rb + j][c],
                    v4 = h[4][rb + j][c];
#pragma unroll
        for (int i = 0; i < kMVR; ++i) {
            const int k = j - i;
            if (k >= 0 && k <= 10) {
                const float w = win.w[k];
                mx[i] = fmaf(w, v0, mx[i]);
                my[i] = fmaf(w, v1, my[i]);
                exx[i] = fmaf(w, v2, exx[i]);
                eyy[i] = fmaf(w, v3, eyy[i]);
                exy[i] = fmaf(w, v4, exy[i]);
            }
        }
    }
    float part = 0.f;
#pragma unroll
    for (int i = 0; i < kMVR; ++i) {
        if (r0 + rb + i >= o.H || c0 + c >= o.W) continue;
        const float sxx = exx[i] - mx[i] * mx[i], syy = eyy[i] - my[i] * my[i], sxy = exy[i] - mx[i] * my[i];
        const float num = (2.f * mx[i] * my[i] + kMC1) * (2.f * sxy + kMC2);
        const float den = (mx[i] * mx[i] + my[i] * my[i] + kMC1) * (sxx + syy + kMC2);
        part += num / den;
    }
    double v = part;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kMetThreads / 32; ++w) t += red[w];
        partials[cta] = t;
    }
}

// T[x][z][y] = A[z][y][x] for both volumes (so that sagittal slices x = const are
// contiguous images with rows z and columns y); 32 x 32 (y, x) tiles through shared
// memory, reads and writes coalesced.
__global__ void __launch_bounds__(256) k_transpose_zyx(const float* __restrict__ a, const float* __restrict__ b,
                                                       int X, int Y, int Z, float* __restrict__ ta,
                                                       float* __restrict__ tb) {
    __shared__ float sa[32][33], sb[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, z = blockIdx.z;
    const long long plane = (long long)z * Y * X;
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int y = y0 + threadIdx.y + k, x = x0 + threadIdx.x;
        if (y < Y && x < X) {
            sa[threadIdx.y + k][threadIdx.x] = a[plane + (long long)y * X + x];
            sb[threadIdx.y + k][threadIdx.x] = b[plane + (long long)y * X + x];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int x = x0 + threadIdx.y + k, y = y0 + threadIdx.x;
        if (y < Y && x < X) {
            const long long o = ((long long)x * Z + z) * Y + y;
            ta[o] = sa[threadIdx.x][threadIdx.y + k];
            tb[o] = sb[threadIdx.x][threadIdx.y + k];
        }
    }
}

__global__ void __launch_bounds__(256) k_sq_err(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                                double* __restrict__ partials) {
    __shared__ double red[8];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float d = a[i] - b[i];
        acc += (double)d * (double)d;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// out = {MSE, PSNR, SSIM (mean of the three), axial, coronal, sagittal}
__global__ void __launch_bounds__(256) k_metrics_fin(const double* __restrict__ tile_partials, Orients os,
                                                     const double* __restrict__ sq_partials, long long n,
                                                     double* __restrict__ out) {
    __shared__ double red[8];
    __shared__ double res[4];
    for (int q = 0; q < 4; ++q) {
        long long lo, hi;
        if (q < 3) {
            lo = os.o[q].first;
            hi = lo + (long long)os.o[q].n * os.o[q].tiles;
        }
        const double* src = q < 3 ? tile_partials : sq_partials;
        if (q == 3) {
            lo = 0;
            hi = kSqBlocks;
        }
        double acc = 0.0;
        for (long long i = lo + threadIdx.x; i < hi; i += 256) acc += src[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red[w];
            res[q] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double ss[3];
        for (int q = 0; q < 3; ++q) ss[q] = res[q] / ((double)os.o[q].n * os.o[q].H * os.o[q].W);
        const double mse = res[3] / (double)n;
        out[0] = mse;
        out[1] = mse > 0.0 ? 10.0 * log10(1.0 / mse) : INFINITY;
        out[2] = (ss[0] + ss[1] + ss[2]) / 3.0;
        out[3] = ss[0];
        out[4] = ss[1];
        out[5] = ss[2];
    }
}

Orients orients(int X, int Y, int Z) {
    const long long XY = (long long)X * Y;
    Orients os;
    os.o[0] = Orient{XY, X, 1, Z, Y, X, 0, 0, 0};   // axial: z = const, rows y, columns x
    os.o[1] = Orient{X, XY, 1, Y, Z, X, 0, 0, 0};   // coronal: y = const, rows z, columns x
    // sagittal: x = const, rows z, columns y -- read from the transposed copies [x][z][y]
    os.o[2] = Orient{(long long)Z * Y, Y, 1, X, Z, Y, 0, 0, 0};
    long long first = 0;
    for (int q = 0; q < 3; ++q) {
        Orient& o = os.o[q];
        o.tiles_x = (o.W + kMT - 1) / kMT;
        o.tiles = o.tiles_x * ((o.H + kMT - 1) / kMT);
        o.first = first;
        first += (long long)o.n * o.tiles;
    }
    return os;
}

long long total_tiles(const Orients& os) { return os.o[2].first + (long long)os.o[2].n * os.o[2].tiles; }

MWin metric_window() {
    double g[11], s = 0;
    for (int k = 0; k < 11; ++k) {
        const double d = k - 5.0;
        g[k] = exp(-d * d / (2 * 1.5 * 1.5));
        s += g[k];
    }
    MWin w;
    for (int k = 0; k < 11; ++k) w.w[k] = (float)(g[k] / s);
    return w;
}

bool bad_dims(int X, int Y, int Z) { return X < 1 || Y < 1 || Z < 1 || X > 4096 || Y > 4096 || Z > 4096; }

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API size_t r2g_metrics_workspace_size(int32_t X, int32_t Y, int32_t Z) {
    if (bad_dims(X, Y, Z)) return 0;
    Layout L;
    L.take(sizeof(double) * (size_t)total_tiles(orients(X, Y, Z)));
    L.take(sizeof(double) * kSqBlocks);
    L.take(sizeof(float) * (size_t)X * Y * Z);
    L.take(sizeof(float) * (size_t)X * Y * Z);
    return L.off;
}

R2G_API r2g_status r2g_volume_metrics(int32_t X, int32_t Y, int32_t Z, const float* vol, const float* ref, double* out,
                                      void* ws, size_t ws_bytes, r2g_stream stream) {
    if (bad_dims(X, Y, Z)) return fail(R2G_E_INVAL, "volume dims must be 1..4096");
    if (!vol || !ref || !out || !ws) return fail(R2G_E_INVAL, "NULL device pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    const Orients os = orients(X, Y, Z);
    const long long nt = total_tiles(os);
    Layout L;
    const size_t o_tiles = L.take(sizeof(double) * (size_t)nt);
    const size_t o_sq = L.take(sizeof(double) * kSqBlocks);
    const size_t o_ta = L.take(sizeof(float) * (size_t)X * Y * Z);
    const size_t o_tb = L.take(sizeof(float) * (size_t)X * Y * Z);
    if (ws_bytes < L.off) return fail(R2G_E_INVAL, "metrics workspace needs %zu bytes", L.off);
    if (nt >= (1ll << 31)) return fail(R2G_E_INVAL, "volume too large");
    char* base = static_cast<char*>(ws);
    double* tp = reinterpret_cast<double*>(base + o_tiles);
    double* sq = reinterpret_cast<double*>(base + o_sq);
    const long long n = (long long)X * Y * Z;
    prof_begin(P_METRICS, stream);
    float* ta = reinterpret_cast<float*>(base + o_ta);
    float* tb = reinterpret_cast<float*>(base + o_tb);
    k_transpose_zyx<<<dim3((unsigned)((X + 31) / 32), (unsigned)((Y + 31) / 32), (unsigned)Z), dim3(32, 8), 0,
                      stream>>>(vol, ref, X, Y, Z, ta, tb);
    k_slice_ssim<<<(unsigned)nt, kMetThreads, 0, stream>>>(vol, ref, ta, tb, os, metric_window(), tp);
    k_sq_err<<<kSqBlocks, 256, 0, stream>>>(vol, ref, n, sq);
    k_metrics_fin<<<1, 256, 0, stream>>>(tp, os, sq, n, out);
    prof_end(P_METRICS, stream);
    note_launches(4);
    return check_launch("r2g_volume_metrics");
}
