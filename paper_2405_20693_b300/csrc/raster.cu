// raster.cu -- the X-ray rasterizer of R^2-Gaussian on sm_103a: projection
// (Eq. 6, Eq. 7, App. A), tile binning, the additive splat (Eq. 5, Eq. 7) and
// its adjoint.
//
// Kernels (all FP32 on the CUDA cores; the path is no dense contraction):
//   k_project      one thread per (view, Gaussian) record: the stated FP32
//                  sequence for p^, Sigma^ and the tile bound, the rectified
//                  amplitude rho_hat = mu rho, and a 32-byte splat record
//                  {cx, cy, A, B, C, rho_hat, rx, ry} in pixel units with the
//                  conic pre-scaled by -log2(e)/2 so that exp(-q/2) = 2^t.
//   emit / sort    (tile, Gaussian id) entries, stable radix sort, tile ranges.
//   k_splat_fwd    one CTA per work item (a tile and a chunk of <= 128 of its
//                  records); records are staged through shared memory; each
//                  lane owns 4 (2 for 8x8 tiles) horizontally adjacent pixels and
//                  accumulates rho_hat 2^t [t >= Tq]; a warp owns an 8-row block
//                  and skips records whose box misses it.  Tiles with several
//                  chunks write per-chunk images; the last chunk to finish sums
//                  them in chunk order.  An empty tile's work item writes zeros.
//   k_splat_bwd    one CTA per work item with dL/dI of the tile in shared
//                  memory; the records' boxes are cut into units of 4 x 2
//                  pixels and the units split evenly over the 128 lanes; each
//                  lane accumulates six moments (sum w, w dx, w dy,
//                  w dx^2, w dx dy, w dy^2; w = g e) of its current record in
//                  registers and adds them with two vector atomics to the
//                  record's slot.
//   k_project_bwd  one thread per Gaussian, looping over views: moments ->
//                  gradients of (rho_hat, p^, conic) -> chain rule through the
//                  projection to d mean, d scale, d quat, d rho.
#include <math.h>

#include "adam_math.cuh"
#include "emit.cuh"
#include "r2g_internal.cuh"

namespace r2g {
namespace {

struct CamF {
    int beam, H, W;
    float L_SD, pu, pv, ou, ov, near_plane;
    int biased;  // 1: rho_hat = rho (no Eq. 7 factor)
    float dil, dil_x, dil_y;  // low-pass dilation (pixels^2) and its detector-unit terms d pu^2, d pv^2
};

struct Params {
    const float* mean;
    const float* scale;
    const float* quat;
    const float* rho;
};

// ------------------------------------------------------------------ stated FP32 projection
// Every step below is one correctly rounded IEEE single operation (the _rn
// intrinsics are never contracted), in the order the header states.

struct Proj {
    float R[3][3];
    float qn[4];
    float qnorm;
    float Mm[3][3];
    float u[3];
    float f, j02, j12;
    float T[2][3];
    float N[2][3];
    float al, be, ga, det;
    float phx, phy;
    bool valid;
};

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

// The operations of the projection: EXACT = the stated sequence (one correctly
// rounded IEEE operation per step, no contraction), else the fast forms.
template <bool EXACT>
struct POps {
    static __device__ __forceinline__ float mul(float a, float b) { return EXACT ? __fmul_rn(a, b) : a * b; }
    static __device__ __forceinline__ float add(float a, float b) { return EXACT ? __fadd_rn(a, b) : a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return EXACT ? __fsub_rn(a, b) : a - b; }
    static __device__ __forceinline__ float div(float a, float b) { return EXACT ? __fdiv_rn(a, b) : a * rcp_fast(b); }
    static __device__ __forceinline__ float sqrt(float x) { return EXACT ? __fsqrt_rn(x) : sqrt_fast(x); }
};

template <bool EXACT>
__device__ __forceinline__ void rotation(const float q[4], Proj& P) {
    using O = POps<EXACT>;
    const auto fm = O::mul;
    const auto fa = O::add;
    const auto fs = O::sub;
    const float n2 = fa(fa(fa(fm(q[0], q[0]), fm(q[1], q[1])), fm(q[2], q[2])), fm(q[3], q[3]));
    const float n = O::sqrt(n2);
    P.qnorm = n;
    const float w = O::div(q[0], n), x = O::div(q[1], n), y = O::div(q[2], n), z = O::div(q[3], n);
    P.qn[0] = w;
    P.qn[1] = x;
    P.qn[2] = y;
    P.qn[3] = z;
    const float xx = fm(x, x), yy = fm(y, y), zz = fm(z, z), xy = fm(x, y), xz = fm(x, z), yz = fm(y, z);
    const float wx = fm(w, x), wy = fm(w, y), wz = fm(w, z);
    P.R[0][0] = fs(1.0f, fm(2.0f, fa(yy, zz)));
    P.R[0][1] = fm(2.0f, fs(xy, wz));
    P.R[0][2] = fm(2.0f, fa(xz, wy));
    P.R[1][0] = fm(2.0f, fa(xy, wz));
    P.R[1][1] = fs(1.0f, fm(2.0f, fa(xx, zz)));
    P.R[1][2] = fm(2.0f, fs(yz, wx));
    P.R[2][0] = fm(2.0f, fs(xz, wy));
    P.R[2][1] = fm(2.0f, fa(yz, wx));
    P.R[2][2] = fs(1.0f, fm(2.0f, fa(xx, yy)));
}

template <bool EXACT = true>
__device__ __forceinline__ void rotation_scale(const float s[3], const float q[4], Proj& P) {
    rotation<EXACT>(q, P);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) P.Mm[j][k] = POps<EXACT>::mul(P.R[j][k], s[k]);
}

// The view-dependent part of the projection, after rotation_scale (R, M) of the
// same Gaussian.
template <bool EXACT = true>
__device__ __forceinline__ void project_view(const float p[3], const float* __restrict__ view, const CamF& cam,
                                             Proj& P) {
    using O = POps<EXACT>;
    const auto fm = O::mul;
    const auto fa = O::add;
    const auto fs = O::sub;
    P.phx = P.phy = P.al = P.be = P.ga = P.det = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        P.u[j] = fa(fa(fa(fm(view[3 * j], p[0]), fm(view[3 * j + 1], p[1])), fm(view[3 * j + 2], p[2])), view[9 + j]);
    P.valid = false;
    if (cam.beam == 1) {
        if (!(P.u[2] > cam.near_plane)) return;
        P.f = O::div(cam.L_SD, P.u[2]);
        P.j02 = -O::div(fm(P.f, P.u[0]), P.u[2]);
        P.j12 = -O::div(fm(P.f, P.u[1]), P.u[2]);
        P.phx = fm(P.f, P.u[0]);
        P.phy = fm(P.f, P.u[1]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P.T[0][k] = fa(fm(P.f, view[k]), fm(P.j02, view[6 + k]));
            P.T[1][k] = fa(fm(P.f, view[3 + k]), fm(P.j12, view[6 + k]));
        }
    } else {
        P.f = 1.0f;
        P.j02 = 0.0f;
        P.j12 = 0.0f;
        P.phx = P.u[0];
        P.phy = P.u[1];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P.T[0][k] = view[k];
            P.T[1][k] = view[3 + k];
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            P.N[a][k] = fa(fa(fm(P.T[a][0], P.Mm[0][k]), fm(P.T[a][1], P.Mm[1][k])), fm(P.T[a][2], P.Mm[2][k]));
    P.al = fa(fa(fm(P.N[0][0], P.N[0][0]), fm(P.N[0][1], P.N[0][1])), fm(P.N[0][2], P.N[0][2]));
    P.be = fa(fa(fm(P.N[0][0], P.N[1][0]), fm(P.N[0][1], P.N[1][1])), fm(P.N[0][2], P.N[1][2]));
    P.ga = fa(fa(fm(P.N[1][0], P.N[1][0]), fm(P.N[1][1], P.N[1][1])), fm(P.N[1][2], P.N[1][2]));
    const float m01 = fs(fm(P.N[0][0], P.N[1][1]), fm(P.N[0][1], P.N[1][0]));
    const float m02 = fs(fm(P.N[0][0], P.N[1][2]), fm(P.N[0][2], P.N[1][0]));
    const float m12 = fs(fm(P.N[0][1], P.N[1][2]), fm(P.N[0][2], P.N[1][1]));
    P.det = fa(fa(fm(m01, m01), fm(m02, m02)), fm(m12, m12));
    if (cam.dil > 0.0f) {
        // optional low-pass dilation: the footprint evaluated at the pixels is
        // Sigma^ + diag(dx, dy); its determinant |Sigma^| + (dy alpha + dx gamma) + dx dy.
        // A constant shift, so the adjoint through (alpha, beta, gamma) is unchanged.
        P.det = fa(fa(P.det, fa(fm(cam.dil_y, P.al), fm(cam.dil_x, P.ga))), fm(cam.dil_x, cam.dil_y));
        P.al = fa(P.al, cam.dil_x);
        P.ga = fa(P.ga, cam.dil_y);
    }
    P.valid = P.det > 0.0f;
}

template <bool EXACT = true>
__device__ __forceinline__ void project_stated(const float p[3], const float s[3], const float q[4],
                                               const float* __restrict__ view, const CamF& cam, Proj& P) {
    rotation_scale<EXACT>(s, q, P);
    project_view<EXACT>(p, view, cam, P);
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

struct Bound {
    float cx, cy, rx, ry;
    int c0, c1, r0, r1;
    bool ok;
};

__device__ __forceinline__ Bound pixel_bound(const Proj& P, const CamF& cam, float Q) {
    Bound b;
    const float ex = __fsqrt_rn(fm(Q, P.al)), ey = __fsqrt_rn(fm(Q, P.ga));
    const float hw = fs(fm(0.5f, (float)cam.W), 0.5f), hh = fs(fm(0.5f, (float)cam.H), 0.5f);
    b.cx = fa(__fdiv_rn(fs(P.phx, cam.ou), cam.pu), hw);
    b.cy = fa(__fdiv_rn(fs(P.phy, cam.ov), cam.pv), hh);
    b.rx = __fdiv_rn(ex, cam.pu);
    b.ry = __fdiv_rn(ey, cam.pv);
    b.c0 = max(0, (int)ceil_clamped(fs(b.cx, b.rx), cam.W));
    b.c1 = min(cam.W - 1, (int)floor_clamped(fa(b.cx, b.rx), cam.W));
    b.r0 = max(0, (int)ceil_clamped(fs(b.cy, b.ry), cam.H));
    b.r1 = min(cam.H - 1, (int)floor_clamped(fa(b.cy, b.ry), cam.H));
    b.ok = P.valid && b.c0 <= b.c1 && b.r0 <= b.r1;
    return b;
}

// omega^T Sigma^{-1} omega with omega the unit source->mean direction (cone) or
// the beam direction (parallel), in the Gaussian's local frame.
__device__ __forceinline__ float kappa_of(const Proj& P, const float s[3], const float* __restrict__ view,
                                          const CamF& cam, float om[3], float v[3]) {
    if (cam.beam == 1) {
        const float il = rsqrtf(P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
        const float n0 = P.u[0] * il, n1 = P.u[1] * il, n2 = P.u[2] * il;
#pragma unroll
        for (int k = 0; k < 3; ++k) om[k] = view[k] * n0 + view[3 + k] * n1 + view[6 + k] * n2;
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) om[k] = view[6 + k];
    }
    float kap = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = P.R[0][k] * om[0] + P.R[1][k] * om[1] + P.R[2][k] * om[2];
        kap += v[k] * v[k] * rcp_fast(s[k] * s[k]);
    }
    return kap;
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

constexpr float kTwoPi = 6.283185307179586f;

// ------------------------------------------------------------------ K1: project

// One record of k_project: the stated FP32 projection, the splat record and the
// tile rectangle (or the debug outputs); returns the record's tile count.
__device__ __forceinline__ uint32_t project_one(const Params& G, const float* __restrict__ views,
                                                const int* __restrict__ view_sel, const CamF& cam, float Q, int TW,
                                                int TH, long long M, long long r, float4* __restrict__ rec,
                                                uint2* __restrict__ rect, float* __restrict__ proj_out,
                                                int* __restrict__ rect_out) {
    const long long v = r / M, i = r - v * M;
    const float* view = views + 12 * (view_sel ? (long long)view_sel[v] : v);
    float p[3], s[3], q[4];
    load_gaussian(G, i, p, s, q);
    Proj P;
    project_stated(p, s, q, view, cam, P);
    const Bound b = pixel_bound(P, cam, Q);
    float rhohat = 0.0f;
    if (b.ok) {
        if (cam.biased) {
            rhohat = G.rho[i];
        } else {
            float om[3], vv[3];
            const float kap = kappa_of(P, s, view, cam, om, vv);
            rhohat = sqrt_fast(kTwoPi * rcp_fast(kap)) * G.rho[i];
        }
    }
    if (rec) {
        float4 a, c;
        if (b.ok) {
            const float id = rcp_fast(P.det);  // the bound above is the stated one; the record need not be
            const float ca = P.ga * id * cam.pu * cam.pu;      // conic in pixel units
            const float cb = -P.be * id * cam.pu * cam.pv;
            const float cc = P.al * id * cam.pv * cam.pv;
            a = make_float4(b.cx, b.cy, -0.5f * kLog2e * ca, -kLog2e * cb);
            c = make_float4(-0.5f * kLog2e * cc, rhohat, b.rx, b.ry);
        } else {
            a = make_float4(0.f, 0.f, 0.f, 0.f);
            c = make_float4(0.f, 0.f, -1.f, -1.f);
        }
        rec[2 * r] = a;
        rec[2 * r + 1] = c;
        uint2 rc;
        if (b.ok) {
            rc.x = (uint32_t)(b.c0 / TW) | ((uint32_t)(b.c1 / TW) << 16);
            rc.y = (uint32_t)(b.r0 / TH) | ((uint32_t)(b.r1 / TH) << 16);
        } else {
            rc.x = 0xffffu;  // lo > hi: no tiles
            rc.y = 0xffffu;
        }
        rect[r] = rc;
    }
    if (proj_out) {
        float* o = proj_out + 8 * r;
        o[0] = P.phx;
        o[1] = P.phy;
        o[2] = P.al;
        o[3] = P.be;
        o[4] = P.ga;
        o[5] = P.det;
        o[6] = rhohat;
        o[7] = b.ok ? 1.0f : 0.0f;
        int* o2 = rect_out + 4 * r;
        o2[0] = b.ok ? b.c0 : 0;
        o2[1] = b.ok ? b.c1 : 0;
        o2[2] = b.ok ? b.r0 : 0;
        o2[3] = b.ok ? b.r1 : 0;
    }
    return b.ok ? (uint32_t)((b.c1 / TW - b.c0 / TW + 1) * (b.r1 / TH - b.r0 / TH + 1)) : 0u;
}

// view_sel (optional, device): view v of this call is views[view_sel[v]].  Each
// thread projects per_thread records, r = ((block * per_thread) + l) * 256 + thread,
// so that a block covers the records of one list block.  mom_clear (optional):
// every record's backward moment slot starts at zero.  lc.partials (optional):
// count the blocks' tile entries for the list build (list_count_tail).
__global__ void __launch_bounds__(256, 4) k_project(Params G, const float* __restrict__ views,
                                                 const int* __restrict__ view_sel, CamF cam, float Q, int TW, int TH,
                                                 long long M, long long n_rec, int per_thread,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 float* __restrict__ proj_out, int* __restrict__ rect_out,
                                                 float4* __restrict__ mom_clear, ListCount lc) {
    unsigned long long cnt = 0;
    for (int l = 0; l < per_thread; ++l) {
        const long long r = ((long long)blockIdx.x * per_thread + l) * 256 + threadIdx.x;
        if (r >= n_rec) continue;
        if (mom_clear) {
            mom_clear[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
            mom_clear[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cnt += project_one(G, views, view_sel, cam, Q, TW, TH, M, r, rec, rect, proj_out, rect_out);
    }
    if (lc.partials) list_count_tail(lc, cnt);
}

// Record r's projection for the cooperative list build (0 entries past n_rec).
struct TileProj {
    Params G;
    const float* views;
    const int* view_sel;
    CamF cam;
    float Q;
    int TW, TH;
    long long M, n_rec;
    float4* rec;
    uint2* rect;
    float4* mom_clear;

    __device__ __forceinline__ uint32_t operator()(long long r) const {
        if (r >= n_rec) return 0u;
        mom_clear[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
        mom_clear[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return project_one(G, views, view_sel, cam, Q, TW, TH, M, r, rec, rect, nullptr, nullptr);
    }
};

// ------------------------------------------------------------------ K2: tile keys

struct TileOp {
    const uint2* rect;
    long long M;
    int tiles_x, tiles_per_view;
    const float4* rec;  // with srec: each sorted entry's splat record is copied next to it
    float4* srec;

    __device__ __forceinline__ void copy_rec(uint64_t x, unsigned long long pos) const {
        if (!srec) return;
        const uint32_t key = (uint32_t)(x >> 32);
        const long long v = key / (uint32_t)tiles_per_view;
        const float4* r = rec + 2 * (size_t)(v * M + (uint32_t)x);
        srec[2 * pos] = r[0];
        srec[2 * pos + 1] = r[1];
    }

    __device__ __forceinline__ uint32_t count(long long r) const {
        const uint2 rc = rect[r];
        const int x0 = rc.x & 0xffff, x1 = rc.x >> 16, y0 = rc.y & 0xffff, y1 = rc.y >> 16;
        return (x1 >= x0 && y1 >= y0) ? (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1)) : 0u;
    }
    // Per-record decode data: x0 | w << 16, y0, key base of the record's view, Gaussian id.
    __device__ __forceinline__ uint4 info(long long r) const {
        const uint2 rc = rect[r];
        const uint32_t x0 = rc.x & 0xffff, x1 = rc.x >> 16;
        const long long v = r / M;
        return make_uint4(x0 | ((x1 - x0 + 1) << 16), rc.y & 0xffff, (uint32_t)(v * tiles_per_view),
                          (uint32_t)(r - v * M));
    }
    // Key of the record's li-th entry (tiles in row-major order of its rectangle).
    __device__ __forceinline__ uint32_t key(const uint4& inf, uint32_t li) const {
        const uint32_t w = inf.x >> 16;
        const uint32_t ty = li / w, tx = li - ty * w;
        return inf.z + (inf.y + ty) * (uint32_t)tiles_x + (inf.x & 0xffff) + tx;
    }
};

// ------------------------------------------------------------------ K3: splat forward

// Pixels per lane of the forward splat for a tile shape (a warp owns an 8-row block
// 4 * PX pixels wide), and the warp blocks per tile.
template <int TW, int TH>
struct FwdShape {
    static constexpr int PX = (TW * TH >= 256) ? 4 : 2;
    static constexpr int BW = 4 * PX;
    static constexpr int NW = TW * TH / (8 * BW);
};
constexpr int kFwdMaxBlocks = 8;   // warp blocks per tile at most (32 x 32 tiles)
constexpr int kFwdWarps = 4;       // independent warps per CTA
constexpr long long kFwdItemWarps = 148ll * 36 * 4;  // work items from which one warp takes a whole item

// Whether the gate of a record can reach a rectangle of pixel centres [x0, x1] x
// [y0, y1] (a superset test: false only when no point of the rectangle has t >=
// Tc, Tc a little below the gate).  t(dx, dy) = A dx^2 + B dx dy + C dy^2 is concave
// with its maximum at the centre, and t(l p) = l^2 t(p) >= t(p) for 0 < l <= 1, so
// when the centre lies outside the rectangle the maximum over it lies on an edge
// whose line separates the two -- at most one vertical and one horizontal edge,
// each maximised over its segment in closed form.  A conic that is not clearly
// negative definite (where FP32 rounding of t could exceed the margin) is always
// kept.  The edge maxima use the approximate reciprocal: near its maximum t is flat
// (an error e in the abscissa changes t by C e^2), far below the margin.
__device__ __forceinline__ bool gate_meets_rect(float4 a, float4 b, float x0, float x1, float y0, float y1,
                                                float Tc) {
    const float A = a.z, B = a.w, C = b.x;
    const float ac4 = 4.0f * A * C;
    if (!(A < 0.0f && C < 0.0f && ac4 - B * B > 0x1p-10f * ac4)) return true;
    const float X0 = x0 - a.x, X1 = x1 - a.x, Y0 = y0 - a.y, Y1 = y1 - a.y;
    const bool inx = X0 <= 0.0f && X1 >= 0.0f, iny = Y0 <= 0.0f && Y1 >= 0.0f;
    if (inx && iny) return true;
    float best = -INFINITY;
    if (!inx) {  // the vertical edge facing the centre: max over dy of C dy^2 + B xe dy + A xe^2
        const float xe = X0 > 0.0f ? X0 : X1;
        const float dy = fminf(fmaxf(-B * xe * rcp_fast(2.0f * C), Y0), Y1);
        best = fmaf(fmaf(A, xe, B * dy), xe, C * dy * dy);
    }
    if (!iny) {  // the horizontal edge facing the centre
        const float ye = Y0 > 0.0f ? Y0 : Y1;
        const float dx = fminf(fmaxf(-B * ye * rcp_fast(2.0f * A), X0), X1);
        best = fmaxf(best, fmaf(fmaf(A, dx, B * ye), dx, C * ye * ye));
    }
    return best >= Tc;
}
// The margin below the gate of the culling test, in units of t (log2 of the
// weight): far above the FP32 rounding of t for the conics it is applied to.
constexpr float kCullMargin = 0.0625f;

// The bounding box of a record's gate inside a rectangle of pixel centres (tile-
// local columns c0..c1, rows r0..r1; centre xc, yc), narrowed in place: columns to
// the x-extent of the gate t >= Tc over the rows, then rows to its y-extent over
// those columns (a superset of the gated pixels for Tc a little below the gate).
// Over a strip of rows the gate's left end bh dy - hh sqrt(K0 - K2 dy^2) is convex
// in dy, its minimum at the row of the gate's leftmost point (dy = B ex / (2C), ex
// its half-width) clamped to the strip; the right end and the y-extent likewise
// (K2 = 4AC - B^2, K0 = 4A Tc, hh = -1 / (2A)).  A conic that is not clearly
// negative definite keeps its box.
__device__ __forceinline__ void narrow_box(float4 a, float4 b, float xc, float yc, float Tc, int& c0, int& c1,
                                           int& r0, int& r1) {
    const float A = a.z, B = a.w, C = b.x;
    const float ac4 = 4.0f * A * C, K2 = ac4 - B * B;
    if (!(A < 0.0f && C < 0.0f && K2 > 0x1p-10f * ac4)) return;
    const float iK2 = rcp_fast(K2);
    {
        const float K0 = 4.0f * A * Tc, hh = -0.5f * rcp_fast(A), bh = B * hh;
        const float ex = sqrt_fast(4.0f * C * Tc * iK2);
        const float dyl = B * ex * (0.5f * rcp_fast(C));
        const float y0 = (float)r0 - yc, y1 = (float)r1 - yc;
        const float dl = fminf(fmaxf(dyl, y0), y1), dr = fminf(fmaxf(-dyl, y0), y1);
        const float xl = fmaf(bh, dl, -sqrt_fast(fmaxf(fmaf(-K2, dl * dl, K0), 0.0f)) * hh);
        const float xr = fmaf(bh, dr, sqrt_fast(fmaxf(fmaf(-K2, dr * dr, K0), 0.0f)) * hh);
        c0 = max(c0, (int)ceilf(xc + xl));
        c1 = min(c1, (int)floorf(xc + xr));
    }
    {
        const float K0 = 4.0f * C * Tc, hh = -0.5f * rcp_fast(C), bh = B * hh;
        const float ey = sqrt_fast(4.0f * A * Tc * iK2);
        const float dxt = B * ey * (0.5f * rcp_fast(A));
        const float x0 = (float)c0 - xc, x1 = (float)c1 - xc;
        const float dt = fminf(fmaxf(dxt, x0), x1), db = fminf(fmaxf(-dxt, x0), x1);
        const float yl = fmaf(bh, dt, -sqrt_fast(fmaxf(fmaf(-K2, dt * dt, K0), 0.0f)) * hh);
        const float yr = fmaf(bh, db, sqrt_fast(fmaxf(fmaf(-K2, db * db, K0), 0.0f)) * hh);
        r0 = max(r0, (int)ceilf(yc + yl));
        r1 = min(r1, (int)floorf(yc + yr));
    }
}

// One warp per (work item, warp block): the item's <= 128 records of one tile are
// read by the warp's lanes (four each), the records whose box and gate meet the
// warp's 8 x BW pixel block are compacted (ballot) into the warp's shared-memory
// list (a record whose gate misses the block would add nothing to it), and
// each lane accumulates its PX pixels over that list -- the quadratic is one FMA per
// pixel (t0 + k (g + A k)).  The warps of a CTA share nothing (no block barrier).
// A tile with several chunks: each chunk's warp writes its block of the chunk image;
// the last chunk of a block to finish (per-(tile, block) arrival counter) sums the
// block's chunk images in chunk order (deterministic).
template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(32 * kFwdWarps, 9) k_splat_fwd(const float4* __restrict__ rec,
                                                              const float4* __restrict__ srec,
                                                              const uint2* __restrict__ ranges,
                                                              const uint64_t* __restrict__ sorted,
                                                              const uint64_t* __restrict__ items,
                                                              const WsStatus* __restrict__ item_st,
                                                              float* __restrict__ partial,
                                                              const uint32_t* __restrict__ item_off,
                                                              uint32_t* __restrict__ key_done, long long M,
                                                              int tiles_x, int tiles_per_view, int H, int W,
                                                              float Tq, float* __restrict__ image, WsStatus* st) {
    constexpr int PX = FwdShape<TW, TH>::PX;  // pixels per lane, along x
    constexpr int BW = FwdShape<TW, TH>::BW;  // warp block: 8 rows x BW columns
    constexpr int NW = FwdShape<TW, TH>::NW;  // warp blocks per tile
    constexpr int WPR = TW / BW;              // warp blocks per tile row
    static_assert(TW % BW == 0 && TH % 8 == 0 && NW <= kFwdMaxBlocks && kChunk == 128, "tile shape");
    __shared__ float4 s_a[kFwdWarps][kChunk];
    __shared__ float4 s_b[kFwdWarps][kChunk];
    pdl_trigger();
    pdl_wait();  // the lists and records of the build before
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long gw = (unsigned long long)blockIdx.x * kFwdWarps + warp;
    const unsigned long long it = gw / NW;
    const int wb = (int)(gw - it * NW);
    // whole warps: past the item count, or after a list build that gave up a wait
    if (it >= item_st->n_keys || st->status == R2G_E_TIMEOUT) return;
    const uint64_t item = items[it];
    const int tile = (int)(item >> 32);
    const uint32_t chunk = (uint32_t)item;
    const int v = tile / tiles_per_view;
    const int lt = tile - v * tiles_per_view;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int bx = (wb % WPR) * BW, by = (wb / WPR) * 8;
    const int lx = bx + (lane & 3) * PX, ly = by + (lane >> 2);
    const int px = tx * TW + lx, py = ty * TH + ly;
    const float fx = (float)px, fy = (float)py;
    const float4* vrec = rec + 2 * (size_t)v * (size_t)M;
    const uint2 rg = ranges[tile];
    const uint32_t start = rg.x + chunk * kChunk;
    const uint32_t end = min(start + (uint32_t)kChunk, rg.y);
    const uint32_t nch = (rg.y - rg.x + kChunk - 1) / kChunk;
    const int n = (int)(end > start ? end - start : 0u);
    // the item's records (lane j holds records j, j + 32, ...), loads issued together:
    // next to the sorted entries (srec), else gathered by Gaussian id
    float4 ra[kChunk / 32], rb[kChunk / 32];
    if (srec) {
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const int j = c * 32 + lane;
            if (j < n) {
                ra[c] = srec[2 * (size_t)(start + j)];      // cx, cy, A, B
                rb[c] = srec[2 * (size_t)(start + j) + 1];  // C, rho_hat, rx, ry
            }
        }
    } else {
        uint32_t gid[kChunk / 32];
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const int j = c * 32 + lane;
            gid[c] = j < n ? (uint32_t)sorted[start + j] : 0u;
        }
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const int j = c * 32 + lane;
            if (j < n) {
                ra[c] = vrec[2 * (size_t)gid[c]];
                rb[c] = vrec[2 * (size_t)gid[c] + 1];
            }
        }
    }
    // compact the records whose pixel box meets this warp's block, in item order
    const int gx0 = tx * TW + bx, gy0 = ty * TH + by;
    int m = 0;
#pragma unroll
    for (int c = 0; c < kChunk / 32; ++c) {
        const int j = c * 32 + lane;
        bool mine = false;
        if (j < n) {
            const float4 a = ra[c], b = rb[c];
            const int c0 = (int)ceilf(a.x - b.z), c1 = (int)floorf(a.x + b.z);
            const int r0 = (int)ceilf(a.y - b.w), r1 = (int)floorf(a.y + b.w);
            mine = c1 >= gx0 && c0 <= gx0 + BW - 1 && r1 >= gy0 && r0 <= gy0 + 7;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, mine);
        if (mine) {
            const int pos = m + __popc(bal & ((1u << lane) - 1u));
            s_a[warp][pos] = ra[c];
            s_b[warp][pos] = rb[c];
        }
        m += __popc(bal);
    }
    __syncwarp();
    // of those, keep the records whose gate meets the block (in place, in order: a
    // kept record moves to a position no later than its own, after its round of 32
    // has been read)
    {
        const int mb = m;
        m = 0;
        for (int q0 = 0; q0 < mb; q0 += 32) {
            const int q = q0 + lane;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            bool keep = false;
            if (q < mb) {
                a = s_a[warp][q];
                b = s_b[warp][q];
                keep = gate_meets_rect(a, b, (float)gx0, (float)(gx0 + BW - 1), (float)gy0, (float)(gy0 + 7),
                                       Tq - kCullMargin);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = m + __popc(bal & ((1u << lane) - 1u));
                s_a[warp][pos] = a;
                s_b[warp][pos] = make_float4(b.x, b.y, 2.0f * a.z, b.w);  // 2A in place of the spent box half-width
            }
            m += __popc(bal);
            __syncwarp();
        }
    }
    float acc[PX];
#pragma unroll
    for (int k = 0; k < PX; ++k) acc[k] = 0.0f;
    unsigned int cnt = 0;
    for (int q = 0; q < m; ++q) {
        const float4 a = s_a[warp][q];
        const float4 b = s_b[warp][q];
        const float dy = fy - a.y;
        const float bdy = a.w * dy;
        const float cdy2 = b.x * dy * dy;
        const float dx0 = fx - a.x;
        // t(dx0 + k) = t0 + k (g + A k), g = dt/ddx at dx0
        const float t0 = fmaf(fmaf(a.z, dx0, bdy), dx0, cdy2);
        const float g = fmaf(b.z, dx0, bdy)  /* b.z = 2A */;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            const float t = k == 0 ? t0 : fmaf((float)k, fmaf(a.z, (float)k, g), t0);
            const float e = ex2_approx(t);
            acc[k] = (t >= Tq) ? fmaf(b.y, e, acc[k]) : acc[k];
            if (COUNT) cnt += (t >= Tq && px + k < W && py < H);
        }
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) atomicAdd(&st->pairs, (unsigned long long)cnt);
    }
    if (nch > 1) {
        // several chunks: store this chunk's block; the last chunk of the block to
        // finish sums the block's chunk images in chunk order
        float* p = partial + it * (size_t)(TW * TH) + ly * TW + lx;
#pragma unroll
        for (int k = 0; k < PX; ++k) p[k] = acc[k];
        __syncwarp();  // every lane's stores ordered before lane 0's release
        uint32_t last = 0;
        if (lane == 0) {
            uint32_t before;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                         : "=r"(before)
                         : "l"(&key_done[(size_t)tile * kFwdMaxBlocks + wb])
                         : "memory");
            last = before == nch - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return;
        __syncwarp();  // lane 0's acquire orders the warp's reads of the other chunks' images
        const float* qp = partial + (size_t)item_off[tile] * (TW * TH) + ly * TW + lx;
#pragma unroll
        for (int k = 0; k < PX; ++k) acc[k] = 0.0f;
        for (uint32_t c = 0; c < nch; ++c)
#pragma unroll
            for (int k = 0; k < PX; ++k) acc[k] += __ldcg(qp + (size_t)c * (TW * TH) + k);
    }
    if (py < H) {  // one chunk (or none: an empty tile's item writes zeros), or the sum
        float* row = image + ((size_t)v * H + py) * W;
#pragma unroll
        for (int k = 0; k < PX; ++k)
            if (px + k < W) row[px + k] = acc[k];
    }
}

// The forward for item counts that fill the GPU several times over (kFwdItemWarps
// and more): one warp per work item.  The item's <= 128 records of one tile are read once by
// the warp's lanes (four each, kept in registers); then for each of the tile's 8 x
// BW pixel blocks in turn, the records whose box and gate meet the block are
// compacted (ballot) into the warp's shared-memory list (a record whose gate misses
// the block would add nothing to it), and each lane accumulates its PX pixels of
// the block over that list -- the quadratic is one FMA per pixel (t0 + k (g + A k)).
// The warps of a CTA share nothing (no block barrier).  A tile with several chunks:
// each chunk writes its blocks of the chunk image; the last chunk of a block to
// finish (per-(tile, block) arrival counter) sums the block's chunk images in chunk
// order (deterministic).
template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(32 * kFwdWarps, 8) k_splat_fwd_items(const float4* __restrict__ rec,
                                                              const float4* __restrict__ srec,
                                                              const uint2* __restrict__ ranges,
                                                              const uint64_t* __restrict__ sorted,
                                                              const uint64_t* __restrict__ items,
                                                              const WsStatus* __restrict__ item_st,
                                                              float* __restrict__ partial,
                                                              const uint32_t* __restrict__ item_off,
                                                              uint32_t* __restrict__ key_done, long long M,
                                                              int tiles_x, int tiles_per_view, int H, int W,
                                                              float Tq, float* __restrict__ image, WsStatus* st) {
    constexpr int PX = FwdShape<TW, TH>::PX;  // pixels per lane, along x
    constexpr int BW = FwdShape<TW, TH>::BW;  // warp block: 8 rows x BW columns
    constexpr int NW = FwdShape<TW, TH>::NW;  // warp blocks per tile
    constexpr int WPR = TW / BW;              // warp blocks per tile row
    static_assert(TW % BW == 0 && TH % 8 == 0 && NW <= kFwdMaxBlocks && kChunk == 128, "tile shape");
    __shared__ float4 s_a[kFwdWarps][kChunk];
    __shared__ float4 s_b[kFwdWarps][kChunk];
    pdl_trigger();
    pdl_wait();  // the lists and records of the build before
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long it = (unsigned long long)blockIdx.x * kFwdWarps + warp;
    // whole warps: past the item count, or after a list build that gave up a wait
    if (it >= item_st->n_keys || st->status == R2G_E_TIMEOUT) return;
    const uint64_t item = items[it];
    const int tile = (int)(item >> 32);
    const uint32_t chunk = (uint32_t)item;
    const int v = tile / tiles_per_view;
    const int lt = tile - v * tiles_per_view;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const float4* vrec = rec + 2 * (size_t)v * (size_t)M;
    const uint2 rg = ranges[tile];
    const uint32_t start = rg.x + chunk * kChunk;
    const uint32_t end = min(start + (uint32_t)kChunk, rg.y);
    const uint32_t nch = (rg.y - rg.x + kChunk - 1) / kChunk;
    const int n = (int)(end > start ? end - start : 0u);
    // the item's records (lane j holds records j, j + 32, ...), loads issued together:
    // next to the sorted entries (srec), else gathered by Gaussian id
    float4 ra[kChunk / 32], rb[kChunk / 32];
    if (srec) {
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const int j = c * 32 + lane;
            if (j < n) {
                ra[c] = srec[2 * (size_t)(start + j)];      // cx, cy, A, B
                rb[c] = srec[2 * (size_t)(start + j) + 1];  // C, rho_hat, rx, ry
            }
        }
    } else {
        uint32_t gid[kChunk / 32];
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const int j = c * 32 + lane;
            gid[c] = j < n ? (uint32_t)sorted[start + j] : 0u;
        }
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const int j = c * 32 + lane;
            if (j < n) {
                ra[c] = vrec[2 * (size_t)gid[c]];
                rb[c] = vrec[2 * (size_t)gid[c] + 1];
            }
        }
    }
    // the tile's blocks each record's gate can reach: its box's blocks, each kept if
    // gate_meets_rect; 8 bits per record (bit by * WPR + bx), the lane's four records
    // in one word
    uint32_t mk = 0;
#pragma unroll
    for (int c = 0; c < kChunk / 32; ++c) {
        const int j = c * 32 + lane;
        if (j < n) {
            const float4 a = ra[c], b = rb[c];
            int c0 = max((int)ceilf(a.x - b.z) - tx * TW, 0), c1 = min((int)floorf(a.x + b.z) - tx * TW, TW - 1);
            int r0 = max((int)ceilf(a.y - b.w) - ty * TH, 0), r1 = min((int)floorf(a.y + b.w) - ty * TH, TH - 1);
            if (c0 <= c1 && r0 <= r1)  // the gate's own bounding box in the tile
                narrow_box(a, b, a.x - (float)(tx * TW), a.y - (float)(ty * TH), Tq - kCullMargin, c0, c1, r0, r1);
            if (c0 <= c1 && r0 <= r1) {
                const int bx0 = c0 / BW, bx1 = c1 / BW, by0 = r0 / 8, by1 = r1 / 8;
                // a convex set whose bounding box spans one row or one column of blocks
                // meets each of them; spanning both, each block is tested
                const bool test = bx1 > bx0 && by1 > by0;
                for (int by = by0; by <= by1; ++by)
                    for (int bx = bx0; bx <= bx1; ++bx) {
                        const float gx0 = (float)(tx * TW + bx * BW), gy0 = (float)(ty * TH + by * 8);
                        if (!test ||
                            gate_meets_rect(a, b, gx0, gx0 + (float)(BW - 1), gy0, gy0 + 7.0f, Tq - kCullMargin))
                            mk |= 1u << (c * 8 + by * WPR + bx);
                    }
            }
        }
    }
    // the box half-widths are spent: the staged records carry 2A in their place
#pragma unroll
    for (int c = 0; c < kChunk / 32; ++c) rb[c].z = 2.0f * ra[c].z;
    for (int wb = 0; wb < NW; ++wb) {
        const int bx = (wb % WPR) * BW, by = (wb / WPR) * 8;
        const int lx = bx + (lane & 3) * PX, ly = by + (lane >> 2);
        const int px = tx * TW + lx, py = ty * TH + ly;
        const float fx = (float)px, fy = (float)py;
        __syncwarp();  // the previous block's list has been read
        // compact the records whose gate meets this block, in item order
        int m = 0;
#pragma unroll
        for (int c = 0; c < kChunk / 32; ++c) {
            const bool mine = (mk >> (c * 8 + wb)) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                const int pos = m + __popc(bal & ((1u << lane) - 1u));
                s_a[warp][pos] = ra[c];
                s_b[warp][pos] = rb[c];
            }
            m += __popc(bal);
        }
        __syncwarp();
        float acc[PX];
#pragma unroll
        for (int k = 0; k < PX; ++k) acc[k] = 0.0f;
        unsigned int cnt = 0;
        for (int q = 0; q < m; ++q) {
            const float4 a = s_a[warp][q];
            const float4 b = s_b[warp][q];
            const float dy = fy - a.y;
            const float bdy = a.w * dy;
            const float cdy2 = b.x * dy * dy;
            const float dx0 = fx - a.x;
            // t(dx0 + k) = t0 + k (g + A k), g = dt/ddx at dx0
            const float t0 = fmaf(fmaf(a.z, dx0, bdy), dx0, cdy2);
            const float g = fmaf(b.z, dx0, bdy)  /* b.z = 2A */;
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                const float t = k == 0 ? t0 : fmaf((float)k, fmaf(a.z, (float)k, g), t0);
                const float e = ex2_approx(t);
                acc[k] = (t >= Tq) ? fmaf(b.y, e, acc[k]) : acc[k];
                if (COUNT) cnt += (t >= Tq && px + k < W && py < H);
            }
        }
        if (COUNT) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (lane == 0 && cnt) atomicAdd(&st->pairs, (unsigned long long)cnt);
        }
        if (nch > 1) {  // several chunks: this chunk's block of the chunk image
            float* p = partial + it * (size_t)(TW * TH) + ly * TW + lx;
#pragma unroll
            for (int k = 0; k < PX; ++k) p[k] = acc[k];
        } else if (py < H) {  // one chunk (or none: an empty tile's item writes zeros)
            float* row = image + ((size_t)v * H + py) * W;
#pragma unroll
            for (int k = 0; k < PX; ++k)
                if (px + k < W) row[px + k] = acc[k];
        }
    }
    if (nch <= 1) return;
    // the item's blocks arrive together (one arrival per block, on lanes 0 .. NW - 1,
    // in one instruction); for each block this chunk was the last to reach, the
    // block's chunk images are summed in chunk order
    __syncwarp();  // every lane's stores ordered before the arriving lanes' release
    uint32_t before = 0;
    const bool arrives = lane < NW;
    if (arrives)
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(before)
                     : "l"(&key_done[(size_t)tile * kFwdMaxBlocks + lane])
                     : "memory");
    const uint32_t lastmask = __ballot_sync(0xffffffffu, arrives && before == nch - 1);
    if (!lastmask) return;
    __syncwarp();  // the arriving lanes' acquire orders the warp's reads of the other chunks' images
    for (int wb = 0; wb < NW; ++wb) {
        if (!((lastmask >> wb) & 1u)) continue;
        const int bx = (wb % WPR) * BW, by = (wb / WPR) * 8;
        const int lx = bx + (lane & 3) * PX, ly = by + (lane >> 2);
        const int px = tx * TW + lx, py = ty * TH + ly;
        const float* qp = partial + (size_t)item_off[tile] * (TW * TH) + ly * TW + lx;
        float acc[PX];
#pragma unroll
        for (int k = 0; k < PX; ++k) acc[k] = 0.0f;
        for (uint32_t c = 0; c < nch; ++c)
#pragma unroll
            for (int k = 0; k < PX; ++k) acc[k] += __ldcg(qp + (size_t)c * (TW * TH) + k);
        if (py < H) {
            float* row = image + ((size_t)v * H + py) * W;
#pragma unroll
            for (int k = 0; k < PX; ++k)
                if (px + k < W) row[px + k] = acc[k];
        }
    }
}

// ------------------------------------------------------------------ K5: splat backward

constexpr int kBwdThreads = 128;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// CTA-wide exclusive scan of one value per thread (kBwdThreads = 128 threads).
__device__ __forceinline__ uint32_t cta_excl_scan_128(uint32_t v, uint32_t* s_w, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(v);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kBwdThreads / 32; ++w) {
        const uint32_t x = s_w[w];
        before += (w < warp) ? x : 0u;
        tot += x;
    }
    *total = tot;
    return before + incl - v;
}

// Backward unit: UW x UH pixels (columns x rows) of a record's box.
constexpr int kBwdUnitW = 4, kBwdUnitH = 2;

// One CTA per work item (<= 128 records of one tile).  Each record's pixel box
// inside the tile, narrowed to the bounding box of its gate there (narrow_box),
// columns c0..c1 and h rows, is cut into ceil(h / UH) rows of
// units of UW x UH pixels whose columns start at multiples of UW (tile-local), so
// that a unit row is one aligned vector load of the staged dL/dI.  A unit may
// reach past the box: those pixels lie outside the box, where the gate t >= Tq
// rejects them exactly as the forward does, or past the tile's last row, where
// the staged dL/dI is padded with UH - 1 zero rows.  The units of the CTA's records are split into
// 128 equal contiguous ranges, one per lane, so every lane evaluates the same
// number of units whatever the record sizes.  A lane derives each unit's row and
// column from its index inside the record (no per-row state, so lanes never
// diverge on row changes), accumulates the six moments of its current record in
// registers, and adds them to the record's slot (two vector atomics) when it
// leaves the record or its range ends.  A lane's range is about one record long,
// so some lane of a warp moves to its next record in most iterations; that branch
// is kept short by staging only the records with units, in consecutive slots, each
// with 2A, 4A, 9A and its Gaussian id.  A unit's second row takes its quadratic
// from the first row's, and the moments are formed once per unit from the two
// rows' sums.
template <int TW, int TH, int UW, int UH>
__global__ void __launch_bounds__(kBwdThreads, 8) k_splat_bwd(const float4* __restrict__ rec,
                                                           const float4* __restrict__ srec,
                                                           const uint2* __restrict__ ranges,
                                                           const uint64_t* __restrict__ sorted,
                                                           const uint64_t* __restrict__ items,
                                                           const WsStatus* __restrict__ item_st, long long M,
                                                           int tiles_x, int tiles_per_view, int H, int W, float Tq,
                                                           const float* __restrict__ dimage,
                                                           float4* __restrict__ mom,
                                                           const WsStatus* __restrict__ st) {
    static_assert(kChunk == kBwdThreads, "one record per thread");
    static_assert(TW <= 32 && TH <= 32 && UW == 4 && UH >= 1 && UH <= 2 && TW % UW == 0,
                  "unit decode is exact for these sizes (units per record <= 2^10); a unit row is one float4");
    constexpr int TWP = TW + 4;           // staged row stride (16-byte multiple; spreads rows over banks)
    constexpr int THP = TH + UH - 1;      // staged rows: UH - 1 zero rows past the tile edge
    __shared__ __align__(16) float s_g[THP * TWP];  // dL/dI of the tile
    // the item's records with units, in item order (empty ones left out, so that a
    // lane's next record is always the next slot)
    __shared__ float4 s_k1[kChunk];        // A, B, C of the conic; dx of the box's first pixel
    __shared__ float4 s_k2[kChunk];        // dy of the first row; s_g index of the first pixel; 1/uw; uw
    __shared__ float4 s_k3[kChunk];        // 2A, 4A, 9A; Gaussian id (bits)
    __shared__ uint32_t s_excl[kChunk + 1];  // exclusive prefix of the unit counts; [records] = total
    __shared__ uint32_t s_w[kBwdThreads / 32];
    pdl_trigger();
    pdl_wait();  // dL/dI of the loss before
    const unsigned long long it = blockIdx.x;
    // past the item count, or after a list build that gave up a wait
    if (it >= item_st->n_keys || st->status == R2G_E_TIMEOUT) return;
    const uint64_t item = items[it];
    const int tile = (int)(item >> 32);
    const uint32_t chunk = (uint32_t)item;
    const int v = tile / tiles_per_view;
    const int lt = tile - v * tiles_per_view;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int X0 = tx * TW, Y0 = ty * TH;
    if ((W & 3) == 0 && (reinterpret_cast<uintptr_t>(dimage) & 15) == 0) {
        // aligned rows: one 16-byte load per 4 pixels (a group lies wholly inside or
        // outside the image); the staged columns past TW are never read
        constexpr int G = TW / 4;
        for (int k = threadIdx.x; k < THP * G; k += kBwdThreads) {
            const int r = k / G, c = 4 * (k - r * G);
            const int gy = Y0 + r, gx = X0 + c;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < TH && gy < H && gx < W)
                val = __ldg(reinterpret_cast<const float4*>(dimage + ((size_t)v * H + gy) * W + gx));
            *reinterpret_cast<float4*>(&s_g[r * TWP + c]) = val;
        }
    } else {
        for (int k = threadIdx.x; k < THP * TWP; k += kBwdThreads) {
            const int r = k / TWP, c = k - r * TWP;
            const int gy = Y0 + r, gx = X0 + c;
            s_g[k] = (r < TH && c < TW && gy < H && gx < W) ? dimage[((size_t)v * H + gy) * W + gx] : 0.0f;
        }
    }
    const uint2 rg = ranges[tile];
    const float4* vrec = rec + 2 * (size_t)v * (size_t)M;
    float4* vmom = mom + 2 * (size_t)v * (size_t)M;
    const int j = threadIdx.x;
    const uint32_t e = rg.x + chunk * kChunk + j;
    uint32_t n = 0;
    float4 K1, K2, K3;
    if (e < rg.y) {
        const uint32_t gid = (uint32_t)sorted[e];
        // the record next to the sorted entry (srec: independent of the id load), else gathered
        const float4 a = srec ? srec[2 * (size_t)e] : vrec[2 * (size_t)gid];
        const float4 b = srec ? srec[2 * (size_t)e + 1] : vrec[2 * (size_t)gid + 1];
        int c0 = max(0, (int)ceilf(a.x - b.z) - X0), c1 = min(TW - 1, (int)floorf(a.x + b.z) - X0);
        int r0 = max(0, (int)ceilf(a.y - b.w) - Y0), r1 = min(TH - 1, (int)floorf(a.y + b.w) - Y0);
        if (c1 >= c0 && r1 >= r0)  // the gate's own bounding box inside the tile
            narrow_box(a, b, a.x - (float)X0, a.y - (float)Y0, Tq - kCullMargin, c0, c1, r0, r1);
        const int w = c1 - c0 + 1, h = r1 - r0 + 1;
        if (w > 0 && h > 0) {
            const int ca = c0 & ~(UW - 1);  // first unit column, aligned
            const int uw = (c1 - ca) / UW + 1;
            n = (uint32_t)(uw * ((h + UH - 1) / UH));
            K1 = make_float4(a.z, a.w, b.x, (float)(X0 + ca) - a.x);
            K2 = make_float4((float)(Y0 + r0) - a.y, (float)(r0 * TWP + ca), 1.0f / (float)uw, (float)uw);
            K3 = make_float4(2.f * a.z, 4.f * a.z, 9.f * a.z, __uint_as_float(gid));
        }
    }
    // one scan of (units | has units << 16) gives the unit offsets and each non-empty
    // record's slot (units per record <= 128, so the low half holds the sum)
    uint32_t T;
    const uint32_t ex = cta_excl_scan_128(n | ((n > 0 ? 1u : 0u) << 16), s_w, &T);
    const int nrec = (int)(T >> 16);
    T &= 0xffffu;
    if (n > 0) {
        const uint32_t slot = ex >> 16;
        s_k1[slot] = K1;
        s_k2[slot] = K2;
        s_k3[slot] = K3;
        s_excl[slot] = ex & 0xffffu;
    }
    if (j == 0) s_excl[nrec] = T;
    __syncthreads();
    const uint32_t per = (T + kBwdThreads - 1) / kBwdThreads;
    const uint32_t p0 = j * per, p1 = min(T, p0 + per);
    if (p0 >= p1) return;
    // the record holding unit p0: the largest k with excl_k <= p0
    int lo = 0, hi = nrec - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_excl[mid] <= p0) lo = mid;
        else hi = mid - 1;
    }
    int k = lo;
    float4 k1 = s_k1[k], k2 = s_k2[k], k3 = s_k3[k];
    uint32_t rec_end = s_excl[k + 1];
    float uf = (float)(p0 - s_excl[k]);  // unit index inside the record
    float S0 = 0.f, Sx = 0.f, Sy = 0.f, Sxx = 0.f, Sxy = 0.f, Syy = 0.f;
    static_assert(UW == 4, "the per-row sums below are written for 4-pixel unit rows");
    // The gate folded into the exponent: with sT = 2^(32 - e), e the exponent of |Tq|,
    // min(t, (t - Tq) sT) is t where t >= Tq; where t < Tq the two differ by at least
    // half an ulp of Tq, 2^(e - 24), so (t - Tq) sT <= -2^8 and 2^min flushes to zero --
    // the pairs of the test t >= Tq (for |Tq| >= 2^-95, i.e. Q >= 4e-29), in two
    // operations and with no select after the multiply by dL/dI.
    const int eT = min(max((int)((__float_as_uint(Tq) >> 23) & 0xffu) - 127, -95), 94);
    const float sT = __uint_as_float((uint32_t)(159 - eT) << 23);
    const float nTq = -Tq * sT;
    const auto gated = [sT, nTq](float t) { return fminf(t, fmaf(t, sT, nTq)); };
    for (uint32_t p = p0; p < p1; ++p) {
        // unit row = floor((u + 1/2) / uw), exact for u < 2^10 and uw <= 16
        const float rowf = floorf(fmaf(uf, k2.z, 0.5f * k2.z));
        const float colf = fmaf(-rowf, k2.w, uf) * (float)UW;  // first pixel column of the unit in the box
        const float dx = k1.w + colf;
        const float dy0 = fmaf(rowf, (float)UH, k2.x);
        const int gi = (int)fmaf(rowf, (float)(UH * TWP), k2.y + colf);
        // the unit's two rows; the second row's t from the first's:
        // t(dx + q, dy + 1) = t(dx + q, dy) + B (dx + q) + C (2 dy + 1)
        // one row's sums of w, q w and q^2 w (its moments at dx + q follow from them)
        const auto row = [&](float t0, float t1, float t2, float t3, const float4 g4, float& W, float& Q1,
                             float& Q2) {
            const float w0 = g4.x * ex2_approx(gated(t0));
            const float w1 = g4.y * ex2_approx(gated(t1));
            const float w2 = g4.z * ex2_approx(gated(t2));
            const float w3 = g4.w * ex2_approx(gated(t3));
            W = (w0 + w1) + (w2 + w3);
            Q1 = fmaf(3.f, w3, fmaf(2.f, w2, w1));
            Q2 = fmaf(9.f, w3, fmaf(4.f, w2, w1));
        };
        static_assert(UH == 2, "two rows per unit");
        const float4 ga = *reinterpret_cast<const float4*>(&s_g[gi]);
        const float4 gb = *reinterpret_cast<const float4*>(&s_g[gi + TWP]);
        const float bdy = k1.y * dy0, cdy2 = k1.z * dy0 * dy0;
        // t(dx + q) = t0 + q gl + A q^2, gl = 2 A dx + B dy
        const float t0 = fmaf(fmaf(k1.x, dx, bdy), dx, cdy2);
        const float gl = fmaf(k3.x, dx, bdy);
        const float t1 = (t0 + k1.x) + gl;
        const float t2 = fmaf(2.f, gl, t0 + k3.y);
        const float t3 = fmaf(3.f, gl, t0 + k3.z);
        float Wa, Q1a, Q2a, Wb, Q1b, Q2b;
        row(t0, t1, t2, t3, ga, Wa, Q1a, Q2a);
        const float d0 = fmaf(k1.y, dx, k1.z * fmaf(2.f, dy0, 1.f)), d1 = d0 + k1.y, d2 = d1 + k1.y;
        row(t0 + d0, t1 + d1, t2 + d2, t3 + (d2 + k1.y), gb, Wb, Q1b, Q2b);
        // the unit's moments, rows dy0 and dy0 + 1: with X = sum w (dx + q),
        // sum w dy = dy0 W + W_b, sum w (dx + q) dy = dy0 X + X_b, sum w dy^2 = dy0 (dy0 W + 2 W_b) + W_b
        const float Wu = Wa + Wb, Q1u = Q1a + Q1b;
        const float Xu = fmaf(Wu, dx, Q1u), Xb = fmaf(Wb, dx, Q1b);
        S0 += Wu;
        Sx += Xu;
        Sxx += fmaf(dx, Xu + Q1u, Q2a + Q2b);  // sum w (dx + q)^2
        Sy += fmaf(Wu, dy0, Wb);
        Sxy += fmaf(Xu, dy0, Xb);
        Syy += fmaf(dy0, fmaf(Wu, dy0, 2.f * Wb), Wb);
        uf += 1.0f;
        if (p + 1 == rec_end && p + 1 < p1) {  // next record
            const size_t g2 = 2 * (size_t)__float_as_uint(k3.w);
            atomicAdd(&vmom[g2], make_float4(S0, Sx, Sy, Sxx));
            atomicAdd(reinterpret_cast<float2*>(&vmom[g2 + 1]), make_float2(Sxy, Syy));
            S0 = Sx = Sy = Sxx = Sxy = Syy = 0.f;
            ++k;
            k1 = s_k1[k];
            k2 = s_k2[k];
            k3 = s_k3[k];
            rec_end = s_excl[k + 1];
            uf = 0.0f;
        }
    }
    const size_t g2 = 2 * (size_t)__float_as_uint(k3.w);
    atomicAdd(&vmom[g2], make_float4(S0, Sx, Sy, Sxx));
    atomicAdd(reinterpret_cast<float2*>(&vmom[g2 + 1]), make_float2(Sxy, Syy));
}

// ------------------------------------------------------------------ K6: projection backward

// dL/dR (full 3x3) -> dL/dq through R(q / |q|).
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
    const float iq = rcp_fast(qnorm);
    dq[0] = (dw - w * dot) * iq;
    dq[1] = (dx - x * dot) * iq;
    dq[2] = (dy - y * dot) * iq;
    dq[3] = (dz - z * dot) * iq;
}

// ADAM: instead of adding the gradients to dmean .. drho, add them to the
// gradient already in adam.grad and take the Adam step of the Gaussian's eleven
// parameters (every Gaussian, with or without moments).
template <bool ADAM>
__global__ void __launch_bounds__(128, 4) k_project_bwd(Params G, const float* __restrict__ views,
                                                     const int* __restrict__ view_sel, CamF cam, float Q,
                                                     long long M, int V, const float4* __restrict__ rec,
                                                     float4* __restrict__ mom, float* __restrict__ dmean,
                                                     float* __restrict__ dscale, float* __restrict__ dquat,
                                                     float* __restrict__ drho, AdamState adam) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    // parameters and Adam moments: written before this step's kernels began
    float p[3], s[3], q[4];
    load_gaussian(G, i, p, s, q);
    const float rho = G.rho[i];
    AdamPre pre;
    if (ADAM) adam_prefetch_state(adam, i, pre);
    pdl_wait();  // the backward moments, and the gradient already in adam.grad
    if (ADAM) {
        adam_prefetch_grad(adam, i, pre);  // issued first: its loads overlap the loss check's
        // a non-finite loss: no update anywhere (every thread sees the same losses); the
        // moments stay in their slots, and the next forward clears them
        if (!adam_loss_ok(adam)) {
            if (i == 0) atomicExch(&adam.guard_status->status, (int32_t)R2G_E_NUMERIC);
            return;
        }
    }
    float gp[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gR[3][3] = {{0.f}}, grho = 0.f;
    float dens_g = 0.f, dens_n = 0.f;  // adaptive-control statistics of this call
    Proj P;
    rotation_scale<false>(s, q, P);  // the Gaussian's R and M, shared by its views
    bool have_rot = false;
    // each view's moments and rho_hat are loaded one view ahead
    float4 n0 = mom[2 * (size_t)i], n1 = mom[2 * (size_t)i + 1];
    float n_rh = rec[2 * (size_t)i + 1].y;
    for (int v = 0; v < V; ++v) {
        const size_t r = (size_t)v * (size_t)M + (size_t)i;
        const float4 m0 = n0, m1 = n1;
        const float rhohat = n_rh;
        if (v + 1 < V) {
            const size_t rn = r + (size_t)M;
            n0 = mom[2 * rn];
            n1 = mom[2 * rn + 1];
            n_rh = rec[2 * rn + 1].y;
        }
        if (m0.x == 0.f && m0.y == 0.f && m0.z == 0.f && m0.w == 0.f && m1.x == 0.f && m1.y == 0.f) continue;
        mom[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);  // consumed: the next backward starts at zero
        mom[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float* view = views + 12 * (view_sel ? view_sel[v] : v);
        project_view<false>(p, view, cam, P);  // values only: no bound is formed here
        have_rot = true;
        // --- moments -> gradients of the pixel-unit record
        const float D = P.det, id = rcp_fast(D);
        const float ca = P.ga * id, cb = -P.be * id, cc = P.al * id;  // conic, detector units
        const float pa = ca * cam.pu * cam.pu, pb = cb * cam.pu * cam.pv, pc = cc * cam.pv * cam.pv;
        const float S0 = m0.x, Sx = m0.y, Sy = m0.z, Sxx = m0.w, Sxy = m1.x, Syy = m1.y;
        const float d_rhohat = S0;
        const float d_cx = rhohat * (pa * Sx + pb * Sy);
        const float d_cy = rhohat * (pb * Sx + pc * Sy);
        const float d_pa = -0.5f * rhohat * Sxx, d_pb = -rhohat * Sxy, d_pc = -0.5f * rhohat * Syy;
        if (adam.dens_grad) {  // |dL/dp^| in normalised device coordinates (pixel gradient x (W/2, H/2))
            dens_g += hypotf(d_cx * (0.5f * (float)cam.W), d_cy * (0.5f * (float)cam.H));
            dens_n += 1.f;
        }
        // --- to detector units
        const float d_phx = d_cx * rcp_fast(cam.pu), d_phy = d_cy * rcp_fast(cam.pv);
        const float d_a = d_pa * cam.pu * cam.pu, d_b = d_pb * cam.pu * cam.pv, d_c = d_pc * cam.pv * cam.pv;
        // --- conic (a, b, c) = (gamma, -beta, alpha) / D  ->  Sigma^ (alpha, beta, gamma)
        const float al = P.al, be = P.be, ga = P.ga, iD2 = id * id;
        const float d_al = (-ga * ga * d_a + be * ga * d_b - be * be * d_c) * iD2;
        const float d_be = (2.f * be * ga * d_a - (al * ga + be * be) * d_b + 2.f * al * be * d_c) * iD2;
        const float d_ga = (-be * be * d_a + al * be * d_b - al * al * d_c) * iD2;
        // --- Sigma^ = N N^T
        float dN[2][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dN[0][k] = 2.f * d_al * P.N[0][k] + d_be * P.N[1][k];
            dN[1][k] = d_be * P.N[0][k] + 2.f * d_ga * P.N[1][k];
        }
        // --- N = T M
        float dT[2][3], dM[3][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) dT[a][j] = dN[a][0] * P.Mm[j][0] + dN[a][1] * P.Mm[j][1] + dN[a][2] * P.Mm[j][2];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) dM[j][k] = P.T[0][j] * dN[0][k] + P.T[1][j] * dN[1][k];
        // --- M = R diag(s)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gR[j][k] += dM[j][k] * s[k];
                gs[k] += dM[j][k] * P.R[j][k];
            }
        // --- rho_hat = mu rho, mu = sqrt(2 pi / kappa) (biased: rho_hat = rho)
        float dom[3] = {0.f, 0.f, 0.f};
        if (cam.biased) {
            grho += d_rhohat;
        } else {
            float om[3], vv[3];
            const float kap = kappa_of(P, s, view, cam, om, vv);
            const float ikap = rcp_fast(kap);
            const float mu = sqrt_fast(kTwoPi * ikap);
            grho += d_rhohat * mu;
            const float d_kap = -0.5f * d_rhohat * rho * mu * ikap;
            float dv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float is = rcp_fast(s[k]), is2 = is * is;
                dv[k] = 2.f * d_kap * vv[k] * is2;
                gs[k] += -2.f * d_kap * vv[k] * vv[k] * is2 * is;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
#pragma unroll
                for (int k = 0; k < 3; ++k) gR[j][k] += om[j] * dv[k];
                dom[j] = P.R[j][0] * dv[0] + P.R[j][1] * dv[1] + P.R[j][2] * dv[2];
            }
        }
        // --- scanner-space mean
        float du[3] = {0.f, 0.f, 0.f};
        if (cam.beam == 1) {
            const float L = cam.L_SD, u0 = P.u[0], u1 = P.u[1], u2 = P.u[2];
            const float iu2 = rcp_fast(u2);
            // T rows: f W0 + j02 W2, f W1 + j12 W2
            float d_f = 0.f, d_j02 = 0.f, d_j12 = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                d_f += dT[0][k] * view[k] + dT[1][k] * view[3 + k];
                d_j02 += dT[0][k] * view[6 + k];
                d_j12 += dT[1][k] * view[6 + k];
            }
            const float f = P.f;
            // f = L/u2, j02 = -L u0/u2^2, j12 = -L u1/u2^2, p^ = (f u0, f u1)
            du[0] += -d_j02 * f * iu2 + d_phx * f;
            du[1] += -d_j12 * f * iu2 + d_phy * f;
            du[2] += -d_f * f * iu2 + 2.f * (d_j02 * u0 + d_j12 * u1) * f * iu2 * iu2 -
                     (d_phx * u0 + d_phy * u1) * f * iu2;
            (void)L;
            // omega = W^T u/|u|
            const float il = rsqrtf(u0 * u0 + u1 * u1 + u2 * u2);
            const float n[3] = {u0 * il, u1 * il, u2 * il};
            float dn[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) dn[j] = view[3 * j] * dom[0] + view[3 * j + 1] * dom[1] + view[3 * j + 2] * dom[2];
            const float nd = n[0] * dn[0] + n[1] * dn[1] + n[2] * dn[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) du[k] += (dn[k] - n[k] * nd) * il;
        } else {
            du[0] += d_phx;
            du[1] += d_phy;
        }
        // --- u = W p + t
#pragma unroll
        for (int k = 0; k < 3; ++k) gp[k] += view[k] * du[0] + view[3 + k] * du[1] + view[6 + k] * du[2];
    }
    float gq[4] = {0.f, 0.f, 0.f, 0.f};
    if (have_rot) quat_grad(P.qn, P.qnorm, gR, gq);
    if (ADAM) {
        const float act[11] = {q[0], q[1], q[2], q[3], p[0], p[1], p[2], s[0], s[1], s[2], rho};
        adam_gaussian_pre(adam, i, pre, act, gq, gp, gs, grho);
        if (adam.dens_grad && dens_n > 0.f) {
            adam.dens_grad[i] += dens_g;
            adam.dens_count[i] += dens_n;
        }
        return;
    }
    if (adam.dens_grad && dens_n > 0.f) {  // an earlier view chunk of a fused step
        adam.dens_grad[i] += dens_g;
        adam.dens_count[i] += dens_n;
    }
    if (!have_rot) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dmean[3 * i + k] += gp[k];
        dscale[3 * i + k] += gs[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) dquat[4 * i + k] += gq[k];
    drho[i] += grho;
}

// Eq. 7's factor mu averaged over the views in front of the near plane; with
// rho_vol, also rho / mean mu (0 where no view keeps the Gaussian).
__global__ void __launch_bounds__(256) k_mean_mu(Params G, const float* __restrict__ views, CamF cam, long long M,
                                                 int V, float* __restrict__ mu_mean, float* __restrict__ rho_vol) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    float p[3], s[3], q[4];
    load_gaussian(G, i, p, s, q);
    float sum = 0.f;
    int n = 0;
    for (int v = 0; v < V; ++v) {
        const float* view = views + 12 * (size_t)v;
        Proj P;
        project_stated(p, s, q, view, cam, P);
        if (cam.beam == 1 && !(P.u[2] > cam.near_plane)) continue;
        float om[3], vv[3];
        sum += sqrtf(kTwoPi / kappa_of(P, s, view, cam, om, vv));
        ++n;
    }
    const float mm = n ? sum / (float)n : 0.f;
    if (mu_mean) mu_mean[i] = mm;
    if (rho_vol) rho_vol[i] = n ? G.rho[i] / mm : 0.f;
}

// ------------------------------------------------------------------ host side

struct RasterLayout {
    size_t status, rec, rect, partials, ranges, key_done, mom, scratch, item_status, item_off, seg, fixed;
    int tiles_x, tiles_y, tiles_per_view;
    long long n_tiles, n_rec;
    SegKeys sk;  // the view-segmented list build, when it applies (several views, > kFusedKeys tiles)
};

// Whether the sorted entries carry their splat records (srec): the fused list build
// copies them during its scatter.  (The view-segmented build does not: at 75 views x
// 500k Gaussians the 32-byte gathers and scattered writes of the copy cost its scatter
// 4 ms for 0.7 ms saved in the forward splat.)
inline bool has_srec(const RasterLayout& L) { return fused_lists(L.n_tiles); }

bool valid_tile(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8) || (tw == 32 && th == 32);
}

r2g_status check_args(int64_t M, int32_t V, const r2g_camera* cam, const r2g_raster_opts* opts) {
    if (!cam || !opts) return fail(R2G_E_INVAL, "camera and options must not be NULL");
    if (M < 1 || M >= (int64_t(1) << 31)) return fail(R2G_E_INVAL, "M = %lld out of range [1, 2^31)", (long long)M);
    if (V < 1) return fail(R2G_E_INVAL, "V = %d must be >= 1", V);
    if ((long long)M * V >= (1ll << 31)) return fail(R2G_E_INVAL, "M * V = %lld must be < 2^31", (long long)M * V);
    if (cam->beam != 0 && cam->beam != 1) return fail(R2G_E_INVAL, "beam must be 0 or 1");
    if (cam->H < 1 || cam->W < 1 || cam->H > 32768 || cam->W > 32768)
        return fail(R2G_E_INVAL, "detector %d x %d out of range", cam->H, cam->W);
    if (!(cam->pitch_u > 0.f) || !(cam->pitch_v > 0.f)) return fail(R2G_E_INVAL, "pitches must be > 0");
    if (cam->beam == 1 && !(cam->L_SD > 0.f)) return fail(R2G_E_INVAL, "cone beam needs L_SD > 0");
    if (!valid_tile(opts->tile_w, opts->tile_h))
        return fail(R2G_E_INVAL, "tile %dx%d not one of 16x16, 8x8, 32x8, 32x32", opts->tile_w, opts->tile_h);
    if (!(opts->Q > 0.f)) return fail(R2G_E_INVAL, "Q must be > 0");
    if (!(opts->dilation >= 0.f) || !(opts->dilation < 1e6f))
        return fail(R2G_E_INVAL, "dilation must be finite and >= 0 (got %g)", (double)opts->dilation);
    if (opts->view_chunk < 0) return fail(R2G_E_INVAL, "view_chunk must be >= 0 (got %d)", opts->view_chunk);
    const long long tx = (cam->W + opts->tile_w - 1) / opts->tile_w, ty = (cam->H + opts->tile_h - 1) / opts->tile_h;
    if ((long long)V * tx * ty >= (1ll << 31)) return fail(R2G_E_INVAL, "too many tiles");
    return R2G_OK;
}

RasterLayout raster_layout(int64_t M, int32_t V, const r2g_camera* cam, const r2g_raster_opts* opts) {
    RasterLayout L;
    L.tiles_x = (cam->W + opts->tile_w - 1) / opts->tile_w;
    L.tiles_y = (cam->H + opts->tile_h - 1) / opts->tile_h;
    L.tiles_per_view = L.tiles_x * L.tiles_y;
    L.n_tiles = (long long)V * L.tiles_per_view;
    L.n_rec = (long long)M * V;
    Layout lay;
    L.status = lay.take(sizeof(WsStatus));
    L.rec = lay.take(32 * (size_t)L.n_rec);
    L.rect = lay.take(8 * (size_t)L.n_rec);
    L.partials = lay.take(8 * (size_t)kScanBlocks);
    L.ranges = lay.take(8 * (size_t)L.n_tiles);
    L.key_done = lay.take(4 * (size_t)L.n_tiles * kFwdMaxBlocks);  // chunk arrivals per (tile, warp block)
    L.item_status = lay.take(sizeof(WsStatus));     // ranges .. item status are cleared together
    L.mom = lay.take(32 * (size_t)L.n_rec);
    L.scratch = lay.take(sort_scratch_bytes());
    L.item_off = lay.take(4 * (size_t)L.n_tiles);
    L.sk = seg_keys(L.n_tiles, M, L.n_rec, L.tiles_per_view);
    L.seg = seg_lists(L.sk) ? lay.take(4 * seg_scratch_words(L.sk)) : 0;
    L.fixed = lay.off;
    return L;
}

// Capacity-dependent tail: two entry buffers, the work items and the per-item
// chunk images of the forward pass.
struct Tail {
    size_t a, b, srec, items, partial, end;
    long long icap;
};

// Fused key spaces also keep each sorted entry's 32-byte splat record next to it
// (srec), so that the splat kernels read records contiguously.
Tail raster_tail(const RasterLayout& L, long long cap, int tile_px) {
    Tail t;
    t.icap = items_capacity(L.n_tiles, cap, kChunk);
    Layout lay;
    lay.off = L.fixed;
    t.a = lay.take(8 * (size_t)cap);
    t.b = lay.take(8 * (size_t)cap);
    t.srec = has_srec(L) ? lay.take(32 * (size_t)cap) : 0;
    t.items = lay.take(8 * (size_t)t.icap);
    t.partial = lay.take(4 * (size_t)tile_px * (size_t)t.icap);
    t.end = lay.off;
    return t;
}

// Largest key capacity (a multiple of 32) whose tail fits in ws_bytes.
long long capacity_of(const RasterLayout& L, size_t ws_bytes, int tile_px) {
    if (ws_bytes <= L.fixed) return 0;
    const double per = (has_srec(L) ? 48.0 : 16.0) + (8.0 + 4.0 * tile_px) / kChunk;
    const double fixed_tail = (double)L.n_tiles * (8.0 + 4.0 * tile_px) + 4096.0;
    double est = ((double)(ws_bytes - L.fixed) - fixed_tail) / per;
    long long cap = est > 0 ? ((long long)est / 32) * 32 : 0;
    if (cap > 0xffffffe0ll) cap = 0xffffffe0ll;
    while (cap + 32 <= 0xffffffe0ll && raster_tail(L, cap + 32, tile_px).end <= ws_bytes) cap += 32;
    while (cap > 0 && raster_tail(L, cap, tile_px).end > ws_bytes) cap -= 32;
    return cap;
}

CamF camf(const r2g_camera* c, const r2g_raster_opts* o) {
    CamF f;
    f.biased = o->biased != 0;
    f.beam = c->beam;
    f.H = c->H;
    f.W = c->W;
    f.L_SD = c->L_SD;
    f.pu = c->pitch_u;
    f.pv = c->pitch_v;
    f.ou = c->off_u;
    f.ov = c->off_v;
    f.near_plane = c->near_plane;
    f.dil = o->dilation > 0.f ? o->dilation : 0.f;
    const float du = f.dil * f.pu, dv = f.dil * f.pv;  // IEEE single products, in this order
    f.dil_x = du * f.pu;
    f.dil_y = dv * f.pv;
    return f;
}

struct FwdArgs {
    const float4* rec;
    const float4* srec;  // the sorted entries' records (fused key spaces), or null
    const uint2* ranges;
    const uint64_t* sorted;
    const uint64_t* items;
    const WsStatus* item_st;
    float* partial;
    const uint32_t* item_off;
    uint32_t* key_done;
};

template <int TW, int TH, bool COUNT>
void fwd_shape(const FwdArgs& f, long long M, const RasterLayout& L, long long icap, int H, int W, float Tq,
               float* image, WsStatus* st, cudaStream_t s) {
    if (FwdShape<TW, TH>::NW > 1 && icap >= kFwdItemWarps) {  // one warp per work item
        launch_pdl(k_splat_fwd_items<TW, TH, COUNT>, dim3((unsigned)((icap + kFwdWarps - 1) / kFwdWarps)),
                   dim3(32 * kFwdWarps), 0, s, f.rec, f.srec, f.ranges, f.sorted, f.items, f.item_st, f.partial,
                   f.item_off, f.key_done, M, L.tiles_x, L.tiles_per_view, H, W, Tq, image, st);
        return;
    }
    const unsigned long long warps = (unsigned long long)icap * FwdShape<TW, TH>::NW;
    launch_pdl(k_splat_fwd<TW, TH, COUNT>, dim3((unsigned)((warps + kFwdWarps - 1) / kFwdWarps)),
               dim3(32 * kFwdWarps), 0, s, f.rec, f.srec, f.ranges, f.sorted, f.items, f.item_st, f.partial,
               f.item_off, f.key_done, M, L.tiles_x, L.tiles_per_view, H, W, Tq, image, st);
}

template <bool COUNT>
void launch_fwd(int tw, int th, const FwdArgs& f, long long M, const RasterLayout& L, long long icap, int H, int W,
                float Tq, float* image, WsStatus* st, cudaStream_t s) {
    if (tw == 16 && th == 16)
        fwd_shape<16, 16, COUNT>(f, M, L, icap, H, W, Tq, image, st, s);
    else if (tw == 8 && th == 8)
        fwd_shape<8, 8, COUNT>(f, M, L, icap, H, W, Tq, image, st, s);
    else if (tw == 32 && th == 32)
        fwd_shape<32, 32, COUNT>(f, M, L, icap, H, W, Tq, image, st, s);
    else
        fwd_shape<32, 8, COUNT>(f, M, L, icap, H, W, Tq, image, st, s);
}

void launch_bwd(int tw, int th, const float4* rec, const float4* srec, const uint2* ranges, const uint64_t* sorted,
                const uint64_t* items, const WsStatus* item_st, long long icap, long long M, const RasterLayout& L,
                int H, int W, float Tq, const float* dimage, float4* mom, const WsStatus* st, cudaStream_t s) {
    const unsigned grid = (unsigned)icap;
#define R2G_BWD(TW, TH)                                                                                       \
    launch_pdl(k_splat_bwd<TW, TH, kBwdUnitW, kBwdUnitH>, dim3(grid), dim3(kBwdThreads), 0, s, rec, srec, ranges, \
               sorted, items, item_st, M, L.tiles_x, L.tiles_per_view, H, W, Tq, dimage, mom, st)
    if (tw == 16 && th == 16)
        R2G_BWD(16, 16);
    else if (tw == 8 && th == 8)
        R2G_BWD(8, 8);
    else if (tw == 32 && th == 32)
        R2G_BWD(32, 32);
    else
        R2G_BWD(32, 8);
#undef R2G_BWD
}

uint64_t* sorted_buffer(char* base, const RasterLayout& L, const Tail& t) {
    return reinterpret_cast<uint64_t*>(base + ((seg_lists(L.sk) || (list_sort_passes(L.n_tiles) & 1)) ? t.b : t.a));
}

// Views per chunk: all V, or opts->view_chunk when it is smaller (the workspace then
// holds one chunk's records and lists).
inline int chunk_views(int V, const r2g_raster_opts* o) { return o->view_chunk > 0 && o->view_chunk < V ? o->view_chunk : V; }

// The workspace carved for a chunk of vc views.
struct Chunk {
    RasterLayout L;
    Tail T;
    long long cap;
    char* base;
    WsStatus* st;
    WsStatus* item_st;
    float4 *rec, *mom, *srec;
    uint2 *rect, *ranges;
    unsigned long long* partials;
    uint32_t *scratch, *item_off, *key_done, *seg;
    uint64_t *a, *b, *items;
    float* partial;
};

bool make_chunk(int64_t M, int vc, const r2g_camera* cam, const r2g_raster_opts* opts, void* ws, size_t ws_bytes,
                Chunk& c) {
    c.L = raster_layout(M, vc, cam, opts);
    const int tpx = opts->tile_w * opts->tile_h;
    c.cap = capacity_of(c.L, ws_bytes, tpx);
    if (c.cap < 32) return false;
    c.T = raster_tail(c.L, c.cap, tpx);
    char* base = static_cast<char*>(ws);
    c.base = base;
    c.st = reinterpret_cast<WsStatus*>(base + c.L.status);
    c.item_st = reinterpret_cast<WsStatus*>(base + c.L.item_status);
    c.rec = reinterpret_cast<float4*>(base + c.L.rec);
    c.mom = reinterpret_cast<float4*>(base + c.L.mom);
    c.srec = has_srec(c.L) ? reinterpret_cast<float4*>(base + c.T.srec) : nullptr;
    c.rect = reinterpret_cast<uint2*>(base + c.L.rect);
    c.ranges = reinterpret_cast<uint2*>(base + c.L.ranges);
    c.partials = reinterpret_cast<unsigned long long*>(base + c.L.partials);
    c.scratch = reinterpret_cast<uint32_t*>(base + c.L.scratch);
    c.item_off = reinterpret_cast<uint32_t*>(base + c.L.item_off);
    c.key_done = reinterpret_cast<uint32_t*>(base + c.L.key_done);
    c.seg = seg_lists(c.L.sk) ? reinterpret_cast<uint32_t*>(base + c.L.seg) : nullptr;
    c.a = reinterpret_cast<uint64_t*>(base + c.T.a);
    c.b = reinterpret_cast<uint64_t*>(base + c.T.b);
    c.items = reinterpret_cast<uint64_t*>(base + c.T.items);
    c.partial = reinterpret_cast<float*>(base + c.T.partial);
    return true;
}

// The records and per-tile lists of one chunk (projection + list build).  first: the
// call's first chunk clears the whole status block; a later chunk clears only the
// arrival counters, so a capacity verdict, the most entries needed and the pair count
// carry over the call's chunks.  Returns the buffer with the sorted entries.
uint64_t* chunk_lists(const Chunk& c, const Params& G, const float* views, const int* view_sel, const CamF& cf,
                      const r2g_raster_opts* opts, long long M, bool first, cudaStream_t stream, int* launches) {
    const RasterLayout& L = c.L;
    if (first)
        cudaMemsetAsync(c.st, 0, sizeof(WsStatus), stream);
    else
        cudaMemsetAsync(&c.st->blocks_done, 0, 2 * sizeof(unsigned long long), stream);  // blocks_done, grid_sync
    TileOp op{c.rect, M, L.tiles_x, L.tiles_per_view, c.rec, c.srec};
    // fused key spaces: projection and lists in one cooperative launch when the grid fits
    const TileProj tp{G, views, view_sel, cf, opts->Q, opts->tile_w, opts->tile_h, M, L.n_rec, c.rec, c.rect, c.mom};
    prof_begin(P_PROJECT, stream);
    if (!opts->separate_lists &&
        launch_plists_coop(tp, op, L.n_rec, L.n_tiles, c.partials, c.a, c.b, c.cap, c.scratch, c.st, c.ranges,
                           c.key_done, c.item_st, c.item_off, c.items, c.T.icap, kChunk, stream, kFwdMaxBlocks)) {
        prof_end(P_PROJECT, stream);
        *launches += 1;
        return c.b;
    }
    const ListBlocking lb = list_blocking(L.n_rec);
    k_project<<<(unsigned)lb.blocks, 256, 0, stream>>>(
        G, views, view_sel, cf, opts->Q, opts->tile_w, opts->tile_h, M, L.n_rec, lb.per_thread, c.rec, c.rect,
        nullptr, nullptr, c.mom,
        c.seg ? seg_list_count(L.sk, c.partials, c.st, c.cap, c.seg)
              : list_count(L.n_tiles, c.partials, c.st, c.cap, c.scratch));
    prof_end(P_PROJECT, stream);
    *launches += 1;
    if (c.seg)
        return build_lists_seg(op, L.n_rec, L.sk, c.partials, c.st, c.a, c.b, c.cap, c.seg, c.ranges, c.key_done,
                               c.item_st, c.item_off, c.items, c.T.icap, kChunk, kFwdMaxBlocks,
                               ListProf{P_EMIT, P_SORT, P_RANGES}, stream, launches);
    return build_lists(op, L.n_rec, L.n_tiles, c.partials, c.st, c.a, c.b, c.scratch, c.cap, c.ranges, c.key_done,
                       c.item_st, c.item_off, c.items, c.T.icap, kChunk, ListProf{P_EMIT, P_SORT, P_RANGES}, stream,
                       launches, !opts->separate_lists, kFwdMaxBlocks);
}

}  // namespace
}  // namespace r2g

using namespace r2g;

R2G_API size_t r2g_raster_workspace_size(int64_t M, int32_t V, const r2g_camera* cam, const r2g_raster_opts* opts,
                                         int64_t key_capacity) {
    if (check_args(M, V, cam, opts) != R2G_OK) return 0;
    if (key_capacity < 1 || key_capacity > 0xffffffe0ll) {
        fail(R2G_E_INVAL, "key_capacity %lld out of range", (long long)key_capacity);
        return 0;
    }
    const RasterLayout L = raster_layout(M, chunk_views(V, opts), cam, opts);
    return raster_tail(L, key_capacity, opts->tile_w * opts->tile_h).end;
}

R2G_API r2g_status r2g_project(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                               int32_t V, const float* views, const r2g_camera* cam, const r2g_raster_opts* opts,
                               float* proj, int32_t* rect, r2g_stream stream) {
    r2g_status e = check_args(M, V, cam, opts);
    if (e) return e;
    if (!mean || !scale || !quat || !rho || !views || !proj || !rect)
        return fail(R2G_E_INVAL, "NULL device pointer");
    if (reinterpret_cast<uintptr_t>(quat) % 16) return fail(R2G_E_INVAL, "quat must be 16-byte aligned");
    const long long n = (long long)M * V;
    Params G{mean, scale, quat, rho};
    k_project<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(G, views, nullptr, camf(cam, opts), opts->Q, opts->tile_w,
                                                                opts->tile_h, M, n, 1, nullptr, nullptr, proj, rect,
                                                                nullptr, ListCount{});
    note_launches(1);
    return check_launch("r2g_project");
}

R2G_API r2g_status r2g_mean_mu(int64_t M, const float* mean, const float* scale, const float* quat,
                               const float* rho, int32_t V, const float* views, const r2g_camera* cam,
                               float* mu_mean, float* rho_vol, r2g_stream stream) {
    r2g_raster_opts o{};
    o.Q = 9.f;
    o.tile_w = o.tile_h = 16;
    r2g_status e = check_args(M, V, cam, &o);
    if (e) return e;
    if (!mean || !scale || !quat || !views) return fail(R2G_E_INVAL, "NULL device pointer");
    if (!mu_mean && !rho_vol) return fail(R2G_E_INVAL, "mu_mean and rho_vol are both NULL");
    if (rho_vol && !rho) return fail(R2G_E_INVAL, "rho_vol needs rho");
    if (reinterpret_cast<uintptr_t>(quat) % 16) return fail(R2G_E_INVAL, "quat must be 16-byte aligned");
    if (M == 0) return R2G_OK;
    Params G{mean, scale, quat, rho};
    k_mean_mu<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>(G, views, camf(cam, &o), M, V, mu_mean, rho_vol);
    note_launches(1);
    return check_launch("r2g_mean_mu");
}

r2g_status r2g::rasterize_impl(int64_t M, const float* mean, const float* scale, const float* quat,
                               const float* rho, int32_t V, const float* views, const int* view_sel,
                               const r2g_camera* cam, const r2g_raster_opts* opts, float* image, void* ws,
                               size_t ws_bytes, cudaStream_t stream) {
    r2g_status e = check_args(M, V, cam, opts);
    if (e) return e;
    if (!mean || !scale || !quat || !rho || !views || !image || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(quat) % 16) return fail(R2G_E_INVAL, "quat must be 16-byte aligned");
    const Params G{mean, scale, quat, rho};
    const CamF cf = camf(cam, opts);
    const float Tq = -0.5f * kLog2e * opts->Q;
    const int Vc = chunk_views(V, opts);
    const size_t px = (size_t)cam->H * cam->W;
    int launches = 0;
    // views c0 .. c0 + vc - 1 at a time (all of them in one chunk unless view_chunk is set)
    for (int c0 = 0; c0 < V; c0 += Vc) {
        const int vc = Vc < V - c0 ? Vc : V - c0;
        Chunk c;
        if (!make_chunk(M, vc, cam, opts, ws, ws_bytes, c))
            return fail(R2G_E_INVAL, "workspace of %zu bytes holds no list entries", ws_bytes);
        const float* views_c = view_sel ? views : views + 12 * (size_t)c0;
        const int* sel_c = view_sel ? view_sel + c0 : nullptr;
        float* image_c = image + (size_t)c0 * px;
        // the radix path gives empty tiles no work item: their pixels stay zero
        if (!fused_lists(c.L.n_tiles) && !seg_lists(c.L.sk))
            cudaMemsetAsync(image_c, 0, sizeof(float) * (size_t)vc * px, stream);
        const uint64_t* sorted = chunk_lists(c, G, views_c, sel_c, cf, opts, M, c0 == 0, stream, &launches);
        prof_begin(P_SPLAT_FWD, stream);
        const FwdArgs fa{c.rec, c.srec, c.ranges, sorted, c.items, c.item_st, c.partial, c.item_off, c.key_done};
        if (opts->count_pairs)
            launch_fwd<true>(opts->tile_w, opts->tile_h, fa, M, c.L, c.T.icap, cam->H, cam->W, Tq, image_c, c.st,
                             stream);
        else
            launch_fwd<false>(opts->tile_w, opts->tile_h, fa, M, c.L, c.T.icap, cam->H, cam->W, Tq, image_c, c.st,
                              stream);
        prof_end(P_SPLAT_FWD, stream);
        launches += 1;
    }
    note_launches(launches);
    return check_launch("r2g_rasterize");
}

R2G_API r2g_status r2g_rasterize(int64_t M, const float* mean, const float* scale, const float* quat,
                                 const float* rho, int32_t V, const float* views, const r2g_camera* cam,
                                 const r2g_raster_opts* opts, float* image, void* ws, size_t ws_bytes,
                                 r2g_stream stream) {
    return rasterize_impl(M, mean, scale, quat, rho, V, views, nullptr, cam, opts, image, ws, ws_bytes, stream);
}

r2g_status r2g::rasterize_backward_impl(int64_t M, const float* mean, const float* scale, const float* quat,
                                        const float* rho, int32_t V, const float* views, const int* view_sel,
                                        const r2g_camera* cam, const r2g_raster_opts* opts, const float* dimage,
                                        float* dmean, float* dscale, float* dquat, float* drho, void* ws,
                                        size_t ws_bytes, cudaStream_t stream, int parts, const AdamState* adam) {
    r2g_status e = check_args(M, V, cam, opts);
    if (e) return e;
    if (!mean || !scale || !quat || !rho || !views || !dimage || !ws) return fail(R2G_E_INVAL, "NULL pointer");
    if (!adam && (!dmean || !dscale || !dquat || !drho)) return fail(R2G_E_INVAL, "NULL gradient pointer");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(R2G_E_INVAL, "workspace must be 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(quat) % 16) return fail(R2G_E_INVAL, "quat must be 16-byte aligned");
    const Params G{mean, scale, quat, rho};
    const CamF cf = camf(cam, opts);
    const float Tq = -0.5f * kLog2e * opts->Q;
    const unsigned grid = (unsigned)((M + 127) / 128);
    const int Vc = chunk_views(V, opts);
    const size_t px = (size_t)cam->H * cam->W;
    const int n_chunks = (V + Vc - 1) / Vc;
    if (n_chunks > 1 && parts != (kRasterBwdMoments | kRasterBwdChain))
        return fail(R2G_E_INVAL, "a view-chunked backward takes the moments and the chain rule together");
    // with an Adam state, the earlier chunks' gradients go to adam->grad and the last
    // chunk's chain rule (the fused one) adds its own and takes the step
    if (adam) {
        dquat = adam->grad ? const_cast<float*>(adam->grad) : nullptr;
        dmean = dquat ? dquat + 4 * M : nullptr;
        dscale = dquat ? dquat + 7 * M : nullptr;
        drho = dquat ? dquat + 10 * M : nullptr;
    }
    int launches = 0;
    // chunks last to first: the last one's records and lists are still in the workspace
    // from the forward; every other chunk's are rebuilt
    for (int ci = n_chunks - 1; ci >= 0; --ci) {
        const int c0 = ci * Vc, vc = Vc < V - c0 ? Vc : V - c0;
        Chunk c;
        if (!make_chunk(M, vc, cam, opts, ws, ws_bytes, c))
            return fail(R2G_E_INVAL, "workspace of %zu bytes holds no list entries", ws_bytes);
        const float* views_c = view_sel ? views : views + 12 * (size_t)c0;
        const int* sel_c = view_sel ? view_sel + c0 : nullptr;
        const uint64_t* sorted =
            ci == n_chunks - 1 ? sorted_buffer(c.base, c.L, c.T)
                               : chunk_lists(c, G, views_c, sel_c, cf, opts, M, false, stream, &launches);
        if (parts & kRasterBwdMoments) {
            prof_begin(P_SPLAT_BWD, stream);
            launch_bwd(opts->tile_w, opts->tile_h, c.rec, c.srec, c.ranges, sorted, c.items, c.item_st, c.T.icap, M,
                       c.L, cam->H, cam->W, Tq, dimage + (size_t)c0 * px, c.mom, c.st, stream);
            prof_end(P_SPLAT_BWD, stream);
            launches += 1;
        }
        if (parts & kRasterBwdChain) {
            prof_begin(P_PROJECT_BWD, stream);
            if (adam && ci == 0) {
                launch_pdl(k_project_bwd<true>, dim3(grid), dim3(128), 0, stream, G, views_c, sel_c, cf, opts->Q, M, vc,
                           c.rec, c.mom, (float*)nullptr, (float*)nullptr, (float*)nullptr, (float*)nullptr, *adam);
            } else {
                // an earlier chunk of a fused step: its gradient (and adaptive-control
                // statistics) are added to what the step accumulates
                AdamState stats{};
                if (adam) {
                    stats.dens_grad = adam->dens_grad;
                    stats.dens_count = adam->dens_count;
                    stats.a.M = M;
                }
                launch_pdl(k_project_bwd<false>, dim3(grid), dim3(128), 0, stream, G, views_c, sel_c, cf, opts->Q, M,
                           vc, c.rec, c.mom, dmean, dscale, dquat, drho, stats);
            }
            prof_end(P_PROJECT_BWD, stream);
            launches += 1;
        }
    }
    note_launches(launches);
    return check_launch("r2g_rasterize_backward");
}

R2G_API r2g_status r2g_rasterize_backward(int64_t M, const float* mean, const float* scale, const float* quat,
                                          const float* rho, int32_t V, const float* views, const r2g_camera* cam,
                                          const r2g_raster_opts* opts, const float* dimage, float* dmean,
                                          float* dscale, float* dquat, float* drho, void* ws, size_t ws_bytes,
                                          r2g_stream stream) {
    return rasterize_backward_impl(M, mean, scale, quat, rho, V, views, nullptr, cam, opts, dimage, dmean, dscale,
                                   dquat, drho, ws, ws_bytes, stream);
}

R2G_API r2g_status r2g_raster_lists(int64_t M, int32_t V, const r2g_camera* cam, const r2g_raster_opts* opts,
                                    const void* ws, size_t ws_bytes, uint32_t* ranges_out, uint32_t* ids,
                                    int64_t capacity, int64_t* n_entries, r2g_stream stream) {
    r2g_status e = check_args(M, V, cam, opts);
    if (e) return e;
    if (!ws || !ranges_out || !ids || !n_entries) return fail(R2G_E_INVAL, "NULL pointer");
    const int Vc = chunk_views(V, opts);
    const RasterLayout L = raster_layout(M, V - ((V - 1) / Vc) * Vc, cam, opts);  // the last chunk's
    const int tpx = opts->tile_w * opts->tile_h;
    const long long cap = capacity_of(L, ws_bytes, tpx);
    if (cap < 32) return fail(R2G_E_INVAL, "workspace of %zu bytes holds no list entries", ws_bytes);
    const Tail T = raster_tail(L, cap, tpx);
    const char* base = static_cast<const char*>(ws);
    WsStatus st;
    if (cudaMemcpyAsync(&st, base + L.status, sizeof(st), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "reading the workspace status failed");
    *n_entries = (int64_t)st.needed;
    if (st.status == R2G_E_CAPACITY) return fail(R2G_E_CAPACITY, "lists overflowed the workspace");
    if ((long long)st.n_keys > capacity) return fail(R2G_E_CAPACITY, "ids buffer too small");
    const uint64_t* sorted = sorted_buffer(const_cast<char*>(base), L, T);
    if (cudaMemcpyAsync(ranges_out, base + L.ranges, 8 * (size_t)L.n_tiles, cudaMemcpyDeviceToDevice, stream) !=
            cudaSuccess ||
        (st.n_keys > 0 &&
         cudaMemcpy2DAsync(ids, 4, sorted, 8, 4, (size_t)st.n_keys, cudaMemcpyDeviceToDevice, stream) !=
             cudaSuccess) ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "copying the lists failed");
    return R2G_OK;
}

