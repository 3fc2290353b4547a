// r2g_oracle.cpp -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
//
// A plain, slow, double-precision CPU statement of what the R^2-Gaussian
// X-ray rasterizer and voxelizer compute (arXiv 2405.20693).  Only the test
// suite, the smoke check and the benchmark's CPU-baseline leg load this file's
// library.  It shares no code, header, table or helper with the CUDA library.
//
// What is here, by the paper's numbering:
//   O1  the method as defined: radiative Gaussians G_i (Eq. 3) with
//       Sigma = R S S^T R^T (Sec. 4.1), the world->scanner transform W, t
//       (App. A), the projective map phi and its local-affine Jacobian J
//       (Eq. 6, App. A, EWA Eq. 29), the rectified 2D Gaussian with amplitude
//       rho_hat = mu * rho, mu = sqrt(2 pi |Sigma~| / |Sigma^|) (Eq. 7), the
//       additive per-pixel sum (Eq. 5, Eq. 7), the density field evaluated on a
//       voxel grid (Eq. 4, Sec. 4.2.2), and hand-derived adjoints of both.
//       The truncation gates q <= Q (pixels) and q <= Q3 (voxels) are part of
//       the definition used here (Sec. 4.2.2 culls at probability 0.99;
//       the rasterizer truncation is the 3-sigma reading).
//   O2  the exact line integral of one 3D Gaussian along a ray (Eq. 1, Eq. 5),
//       no truncation.
//   O3  trapezoid quadrature of the same integral (a brute-force pin for O2).
//   R32 an FP32 replica of the stated projection-and-tile-bound op sequence,
//       so that per-tile Gaussian lists can be compared bit for bit.
//
// Parameter kinds throughout: mean[M][3], scale[M][3] (positive, already
// activated), quat[M][4] (w, x, y, z; normalised here), rho[M].
// Views: an FP32 table [V][12] = W (3x3 row-major) then t (3), widened to
// double.  Detector pixel (r, c) has its centre at
//   xi  = (c + 1/2 - W/2) * pitch_u + off_u,   eta = (r + 1/2 - H/2) * pitch_v + off_v
// in scanner-plane units; rows run along the scanner's second axis.
//
// Everything is single-threaded and obvious on purpose.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

using cd = std::complex<double>;

inline double re(double x) { return x; }
inline double re(const cd& x) { return x.real(); }

struct Cam {
    int beam;        // 0 = parallel, 1 = cone
    int H, W;        // detector rows, columns
    double L_SD;     // source-to-detector distance (cone)
    double pitch_u, pitch_v, off_u, off_v;
    double near_plane;  // cone: drop Gaussians with u2 <= near_plane
    int jmode;          // third Jacobian row: 0 = u/|u| (EWA, used everywhere);
                        // 1 = (0, 0, 1), a planted mistake for the reading test only
    int biased;         // 1 = the X-3DGS amplitude rho_hat = rho (no integration bias
                        // correction, Sec. 4.2.1); 0 = the rectified rho_hat = mu rho (Eq. 7)
    double dilation;    // low-pass dilation in pixels^2 (0 = none): the footprint evaluated at
                        // the pixels is Sigma^ + dilation diag(pitch_u^2, pitch_v^2), as 3DGS
                        // does for anti-aliasing; mu (Eq. 7) keeps the undilated Sigma^
};

template <class T> struct M3 { T a[3][3]; };

template <class T> M3<T> mul(const M3<T>& A, const M3<T>& B) {
    M3<T> C;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T s = 0;
            for (int k = 0; k < 3; ++k) s += A.a[i][k] * B.a[k][j];
            C.a[i][j] = s;
        }
    return C;
}
template <class T> M3<T> transpose(const M3<T>& A) {
    M3<T> C;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[j][i];
    return C;
}
template <class T> T det3(const M3<T>& A) {
    const auto& a = A.a;
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
           a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}
// cofactor matrix: cof[i][j] = (-1)^(i+j) * minor(i, j); inverse = cof^T / det
template <class T> M3<T> cofactor(const M3<T>& A) {
    const auto& a = A.a;
    M3<T> C;
    C.a[0][0] = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    C.a[0][1] = -(a[1][0] * a[2][2] - a[1][2] * a[2][0]);
    C.a[0][2] = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    C.a[1][0] = -(a[0][1] * a[2][2] - a[0][2] * a[2][1]);
    C.a[1][1] = a[0][0] * a[2][2] - a[0][2] * a[2][0];
    C.a[1][2] = -(a[0][0] * a[2][1] - a[0][1] * a[2][0]);
    C.a[2][0] = a[0][1] * a[1][2] - a[0][2] * a[1][1];
    C.a[2][1] = -(a[0][0] * a[1][2] - a[0][2] * a[1][0]);
    C.a[2][2] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
    return C;
}
template <class T> M3<T> inverse(const M3<T>& A) {
    M3<T> C = transpose(cofactor(A));
    T d = det3(A);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C.a[i][j] /= d;
    return C;
}

// Rotation matrix of the unit quaternion (w, x, y, z) (Sec. 4.1 follows 3DGS).
template <class T> M3<T> quat_to_R(T w, T x, T y, T z) {
    M3<T> R;
    R.a[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R.a[0][1] = 2.0 * (x * y - w * z);
    R.a[0][2] = 2.0 * (x * z + w * y);
    R.a[1][0] = 2.0 * (x * y + w * z);
    R.a[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R.a[1][2] = 2.0 * (y * z - w * x);
    R.a[2][0] = 2.0 * (x * z - w * y);
    R.a[2][1] = 2.0 * (y * z + w * x);
    R.a[2][2] = 1.0 - 2.0 * (x * x + y * y);
    return R;
}

// Sigma = R S S^T R^T with S = diag(s) and R from the normalised quaternion.
template <class T> void covariance(const T* s, const T* q, M3<T>& Sigma, M3<T>& R, T qn[4], T& qnorm) {
    qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) qn[k] = q[k] / qnorm;
    R = quat_to_R(qn[0], qn[1], qn[2], qn[3]);
    M3<T> S{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S.a[i][j] = (i == j) ? s[i] : T(0);
    M3<T> RS = mul(R, S);
    Sigma = mul(RS, transpose(RS));
}

// One Gaussian seen from one view (Eq. 6, Eq. 7, App. A).
template <class T> struct Proj {
    bool valid;
    T u[3];          // scanner-space mean, u = W p + t
    M3<T> J;         // Jacobian of phi at u
    M3<T> A;         // J W
    M3<T> St;        // Sigma~ = J W Sigma W^T J^T
    T sh[3];         // Sigma^ = top-left 2x2 of Sigma~: (alpha, beta, gamma)
    T d3, d2;        // |Sigma~|, |Sigma^|
    T shd[3];        // the evaluated footprint: Sigma^ plus the dilation (= sh without one)
    T mu, rhohat;    // mu = sqrt(2 pi d3 / d2), rho_hat = mu rho
    T ph[2];         // p^ = first two coordinates of phi(u)
    T conic[3];      // Sigma^^{-1} = [[a, b], [b, c]]
};

template <class T>
Proj<T> project_one(const T* p, const M3<T>& Sigma, T rho, const double* view, const Cam& cam) {
    Proj<T> P{};
    M3<T> Wm;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Wm.a[i][j] = view[3 * i + j];
    for (int i = 0; i < 3; ++i) P.u[i] = Wm.a[i][0] * p[0] + Wm.a[i][1] * p[1] + Wm.a[i][2] * p[2] + view[9 + i];
    const T u0 = P.u[0], u1 = P.u[1], u2 = P.u[2];
    P.valid = true;
    if (cam.beam == 1) {
        if (re(u2) <= cam.near_plane) { P.valid = false; return P; }
        // phi(u) = (L u0/u2, L u1/u2, |u|): the pinhole map in detector units with the
        // ray-space depth |u| (EWA); J is its derivative.
        const double L = cam.L_SD;
        const T l = std::sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        P.J.a[0][0] = L / u2; P.J.a[0][1] = 0.0; P.J.a[0][2] = -L * u0 / (u2 * u2);
        P.J.a[1][0] = 0.0; P.J.a[1][1] = L / u2; P.J.a[1][2] = -L * u1 / (u2 * u2);
        if (cam.jmode == 1) {
            P.J.a[2][0] = 0.0; P.J.a[2][1] = 0.0; P.J.a[2][2] = 1.0;
        } else {
            P.J.a[2][0] = u0 / l; P.J.a[2][1] = u1 / l; P.J.a[2][2] = u2 / l;
        }
        P.ph[0] = L * u0 / u2;
        P.ph[1] = L * u1 / u2;
    } else {
        // parallel beam (the L_SO -> infinity limit): phi = identity, J = I
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) P.J.a[i][j] = (i == j) ? 1.0 : 0.0;
        P.ph[0] = u0;
        P.ph[1] = u1;
    }
    P.A = mul(P.J, Wm);
    P.St = mul(mul(P.A, Sigma), transpose(P.A));
    P.sh[0] = P.St.a[0][0];
    P.sh[1] = P.St.a[0][1];
    P.sh[2] = P.St.a[1][1];
    P.d3 = det3(P.St);
    P.d2 = P.sh[0] * P.sh[2] - P.sh[1] * P.sh[1];
    if (!(re(P.d2) > 0.0)) { P.valid = false; return P; }
    P.mu = std::sqrt(2.0 * M_PI * P.d3 / P.d2);
    P.rhohat = cam.biased ? rho : P.mu * rho;
    // the footprint evaluated at the pixels (optional low-pass dilation; a constant
    // added to Sigma^, so d footprint / d Sigma^ is the identity)
    P.shd[0] = P.sh[0] + cam.dilation * cam.pitch_u * cam.pitch_u;
    P.shd[1] = P.sh[1];
    P.shd[2] = P.sh[2] + cam.dilation * cam.pitch_v * cam.pitch_v;
    const T dd = P.shd[0] * P.shd[2] - P.shd[1] * P.shd[1];
    P.conic[0] = P.shd[2] / dd;
    P.conic[1] = -P.shd[1] / dd;
    P.conic[2] = P.shd[0] / dd;
    return P;
}

inline double pix_xi(int c, const Cam& cam) { return (c + 0.5 - 0.5 * cam.W) * cam.pitch_u + cam.off_u; }
inline double pix_eta(int r, const Cam& cam) { return (r + 0.5 - 0.5 * cam.H) * cam.pitch_v + cam.off_v; }

// Inclusive index range of pixel centres within |centre - m| <= e, widened by one
// pixel on each side (the gate decides membership; the widening only guards
// rounding at the edge of the exact bounding box).
inline void centre_range(double m, double e, double pitch, double off, int n, int& lo, int& hi) {
    if (!std::isfinite(e)) { lo = 0; hi = n - 1; return; }
    const double a = (m - e - off) / pitch + 0.5 * n - 0.5;
    const double b = (m + e - off) / pitch + 0.5 * n - 0.5;
    lo = (int)std::max(-1.0, std::min((double)n, std::ceil(a) - 1.0));
    hi = (int)std::max(-1.0, std::min((double)n, std::floor(b) + 1.0));
    lo = std::max(lo, 0);
    hi = std::min(hi, n - 1);
}

struct Params {
    int64_t M;
    const double *mean, *scale, *quat, *rho;
};

template <class T> struct ParamsT {
    std::vector<T> mean, scale, quat, rho;
};

template <class T> ParamsT<T> widen(const Params& P) {
    ParamsT<T> Q;
    Q.mean.assign(P.mean, P.mean + 3 * P.M);
    Q.scale.assign(P.scale, P.scale + 3 * P.M);
    Q.quat.assign(P.quat, P.quat + 4 * P.M);
    Q.rho.assign(P.rho, P.rho + P.M);
    return Q;
}

// O1 rasterizer: I[v, r, c] = sum_i rho_hat_i exp(-q/2) [q <= Q], scatter form
// (each Gaussian visits the pixels of its exact bounding box; identical to the
// all-pixels sum because the box holds every pixel with q <= Q).
// band (optional): per pixel, the summed |rho_hat| e^{-q/2} of Gaussians whose q is
// within 1e-4 Q of the gate (the pixels where an FP32 q may decide otherwise).
template <class T>
int64_t render(const ParamsT<T>& G, int64_t M, const double* views, int V, const Cam& cam, double Q,
               T* img, double* band, bool brute) {
    const int H = cam.H, Wd = cam.W;
    for (int64_t k = 0; k < (int64_t)V * H * Wd; ++k) img[k] = 0.0;
    if (band)
        for (int64_t k = 0; k < (int64_t)V * H * Wd; ++k) band[k] = 0.0;
    int64_t pairs = 0;
    for (int v = 0; v < V; ++v) {
        const double* view = views + 12 * v;
        T* Iv = img + (int64_t)v * H * Wd;
        for (int64_t i = 0; i < M; ++i) {
            M3<T> Sigma, R;
            T qn[4], qnorm;
            covariance(&G.scale[3 * i], &G.quat[4 * i], Sigma, R, qn, qnorm);
            Proj<T> P = project_one(&G.mean[3 * i], Sigma, G.rho[i], view, cam);
            if (!P.valid) continue;
            int c0 = 0, c1 = Wd - 1, r0 = 0, r1 = H - 1;
            if (!brute) {
                centre_range(re(P.ph[0]), std::sqrt(Q * re(P.shd[0])), cam.pitch_u, cam.off_u, Wd, c0, c1);
                centre_range(re(P.ph[1]), std::sqrt(Q * re(P.shd[2])), cam.pitch_v, cam.off_v, H, r0, r1);
            }
            for (int r = r0; r <= r1; ++r) {
                const T dy = pix_eta(r, cam) - P.ph[1];
                for (int c = c0; c <= c1; ++c) {
                    const T dx = pix_xi(c, cam) - P.ph[0];
                    const T q = P.conic[0] * dx * dx + 2.0 * P.conic[1] * dx * dy + P.conic[2] * dy * dy;
                    const double qr = re(q);
                    if (band && std::fabs(qr - Q) <= 1e-4 * Q)
                        band[(int64_t)v * H * Wd + (int64_t)r * Wd + c] +=
                            std::fabs(re(P.rhohat)) * std::exp(-0.5 * qr);
                    if (!(qr <= Q)) continue;
                    Iv[(int64_t)r * Wd + c] += P.rhohat * std::exp(-0.5 * q);
                    ++pairs;
                }
            }
        }
    }
    return pairs;
}

// O1 rasterizer with the gate of every Gaussian held at a second parameter set Gg:
// the box and the pixels with q <= Q come from Gaussian i of Gg, the value
// rho_hat e^{-q/2} at those pixels from Gaussian i of G.  With G == Gg this is
// render().  A central difference in G is then the derivative with the gate
// membership fixed -- the quantity an adjoint of the gated sum computes (the gate's
// moving boundary adds jumps of e^{-Q/2} rho_hat that no derivative sees).
int64_t render_gated(const ParamsT<double>& G, const ParamsT<double>& Gg, int64_t M, const double* views, int V,
                     const Cam& cam, double Q, double* img) {
    const int H = cam.H, Wd = cam.W;
    for (int64_t k = 0; k < (int64_t)V * H * Wd; ++k) img[k] = 0.0;
    int64_t pairs = 0;
    for (int v = 0; v < V; ++v) {
        const double* view = views + 12 * v;
        double* Iv = img + (int64_t)v * H * Wd;
        for (int64_t i = 0; i < M; ++i) {
            M3<double> Sg, Rg, S, R;
            double qg[4], ng, qn[4], nn;
            covariance(&Gg.scale[3 * i], &Gg.quat[4 * i], Sg, Rg, qg, ng);
            covariance(&G.scale[3 * i], &G.quat[4 * i], S, R, qn, nn);
            const Proj<double> Pg = project_one(&Gg.mean[3 * i], Sg, Gg.rho[i], view, cam);
            const Proj<double> P = project_one(&G.mean[3 * i], S, G.rho[i], view, cam);
            if (!Pg.valid || !P.valid) continue;
            int c0, c1, r0, r1;
            centre_range(Pg.ph[0], std::sqrt(Q * Pg.shd[0]), cam.pitch_u, cam.off_u, Wd, c0, c1);
            centre_range(Pg.ph[1], std::sqrt(Q * Pg.shd[2]), cam.pitch_v, cam.off_v, H, r0, r1);
            for (int r = r0; r <= r1; ++r) {
                const double eta = pix_eta(r, cam);
                for (int c = c0; c <= c1; ++c) {
                    const double xi = pix_xi(c, cam);
                    const double gx = xi - Pg.ph[0], gy = eta - Pg.ph[1];
                    const double qgate = Pg.conic[0] * gx * gx + 2.0 * Pg.conic[1] * gx * gy + Pg.conic[2] * gy * gy;
                    if (!(qgate <= Q)) continue;
                    const double dx = xi - P.ph[0], dy = eta - P.ph[1];
                    const double q = P.conic[0] * dx * dx + 2.0 * P.conic[1] * dx * dy + P.conic[2] * dy * dy;
                    Iv[(int64_t)r * Wd + c] += P.rhohat * std::exp(-0.5 * q);
                    ++pairs;
                }
            }
        }
    }
    return pairs;
}

// ---------------------------------------------------------------------------
// Hand-derived adjoint of the O1 rasterizer.  Gradients are accumulated (+=).
// Matrix gradients are taken entry-wise on full (not symmetrised) matrices.

struct Grad {
    double* mean;
    double* scale;
    double* quat;
    double* rho;
};

// dL/dR (full 3x3) of R(qn) -> dL/dqn, then through qn = q/|q|.
void quat_backward(const double qn[4], double qnorm, const M3<double>& dR, double* dq) {
    const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    const auto& g = dR.a;
    double dw = 0, dx = 0, dy = 0, dz = 0;
    // R00 = 1 - 2(y^2 + z^2)
    dy += -4 * y * g[0][0]; dz += -4 * z * g[0][0];
    // R01 = 2(xy - wz)
    dx += 2 * y * g[0][1]; dy += 2 * x * g[0][1]; dw += -2 * z * g[0][1]; dz += -2 * w * g[0][1];
    // R02 = 2(xz + wy)
    dx += 2 * z * g[0][2]; dz += 2 * x * g[0][2]; dw += 2 * y * g[0][2]; dy += 2 * w * g[0][2];
    // R10 = 2(xy + wz)
    dx += 2 * y * g[1][0]; dy += 2 * x * g[1][0]; dw += 2 * z * g[1][0]; dz += 2 * w * g[1][0];
    // R11 = 1 - 2(x^2 + z^2)
    dx += -4 * x * g[1][1]; dz += -4 * z * g[1][1];
    // R12 = 2(yz - wx)
    dy += 2 * z * g[1][2]; dz += 2 * y * g[1][2]; dw += -2 * x * g[1][2]; dx += -2 * w * g[1][2];
    // R20 = 2(xz - wy)
    dx += 2 * z * g[2][0]; dz += 2 * x * g[2][0]; dw += -2 * y * g[2][0]; dy += -2 * w * g[2][0];
    // R21 = 2(yz + wx)
    dy += 2 * z * g[2][1]; dz += 2 * y * g[2][1]; dw += 2 * x * g[2][1]; dx += 2 * w * g[2][1];
    // R22 = 1 - 2(x^2 + y^2)
    dx += -4 * x * g[2][2]; dy += -4 * y * g[2][2];
    const double dqn[4] = {dw, dx, dy, dz};
    const double dot = qn[0] * dqn[0] + qn[1] * dqn[1] + qn[2] * dqn[2] + qn[3] * dqn[3];
    for (int k = 0; k < 4; ++k) dq[k] += (dqn[k] - qn[k] * dot) / qnorm;
}

// dL/dSigma (full) with Sigma = R diag(s^2) R^T -> dL/ds, dL/dq.
void sigma_backward(const M3<double>& dSigma, const M3<double>& R, const double* s, const double qn[4],
                    double qnorm, double* ds, double* dq) {
    M3<double> Gs;  // dSigma + dSigma^T
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Gs.a[i][j] = dSigma.a[i][j] + dSigma.a[j][i];
    M3<double> D{};
    for (int k = 0; k < 3; ++k) D.a[k][k] = s[k] * s[k];
    // dR = (dSigma + dSigma^T) R D
    M3<double> dR = mul(mul(Gs, R), D);
    // dD_kk = (R^T dSigma R)_kk, D_kk = s_k^2
    M3<double> RtGR = mul(mul(transpose(R), dSigma), R);
    for (int k = 0; k < 3; ++k) ds[k] += 2.0 * s[k] * RtGR.a[k][k];
    quat_backward(qn, qnorm, dR, dq);
}

// Chain rule from the record gradient drec = d(rho_hat, p^x, p^y, a, b, c) of one
// (Gaussian, view) to the parameters of Gaussian i (accumulated into g).
void chain_record(const Proj<double>& P, const M3<double>& Sigma, const M3<double>& R, const double qn[4],
                  double qnorm, const M3<double>& Wm, const Cam& cam, const ParamsT<double>& G, int64_t i,
                  const double drec[6], Grad g, int64_t oi) {
    const double d_rhohat = drec[0], d_ph0 = drec[1], d_ph1 = drec[2], da = drec[3], db = drec[4], dc = drec[5];
    const double a = P.conic[0], b = P.conic[1], c = P.conic[2];
    // rho_hat = mu rho (rectified, Eq. 7) or rho_hat = rho (X-3DGS, no mu term)
    g.rho[oi] += cam.biased ? d_rhohat : d_rhohat * P.mu;
    const double dmu = cam.biased ? 0.0 : d_rhohat * G.rho[i];
    // mu = sqrt(2 pi d3 / d2)
    const double dd3 = dmu * P.mu / (2.0 * P.d3);
    const double dd2 = -dmu * P.mu / (2.0 * P.d2);
    // conic = (Sigma^ + dilation)^{-1}: full-matrix gradient Gc = [[da, db/2], [db/2, dc]];
    // dL/dSigma^ = -C Gc C with C the conic (the dilation is a constant).
    const double C2[2][2] = {{a, b}, {b, c}};
    const double Gc[2][2] = {{da, 0.5 * db}, {0.5 * db, dc}};
    double T1[2][2], dSh[2][2];
    for (int p = 0; p < 2; ++p)
        for (int q2 = 0; q2 < 2; ++q2) T1[p][q2] = C2[p][0] * Gc[0][q2] + C2[p][1] * Gc[1][q2];
    for (int p = 0; p < 2; ++p)
        for (int q2 = 0; q2 < 2; ++q2) dSh[p][q2] = -(T1[p][0] * C2[0][q2] + T1[p][1] * C2[1][q2]);
    // d2 = |Sigma^|: d d2 / d Sigma^ = cofactor(Sigma^) = [[gamma, -beta], [-beta, alpha]]
    dSh[0][0] += dd2 * P.sh[2];
    dSh[1][1] += dd2 * P.sh[0];
    dSh[0][1] += -dd2 * P.sh[1];
    dSh[1][0] += -dd2 * P.sh[1];
    // Sigma~ gradient: top-left block from Sigma^, plus d3 = |Sigma~| (cofactor)
    M3<double> dSt{};
    for (int p = 0; p < 2; ++p)
        for (int q2 = 0; q2 < 2; ++q2) dSt.a[p][q2] += dSh[p][q2];
    M3<double> cof = cofactor(P.St);
    for (int p = 0; p < 3; ++p)
        for (int q2 = 0; q2 < 3; ++q2) dSt.a[p][q2] += dd3 * cof.a[p][q2];
    // Sigma~ = A Sigma A^T:  dA = (G + G^T) A Sigma,  dSigma = A^T G A
    M3<double> Gs2;
    for (int p = 0; p < 3; ++p)
        for (int q2 = 0; q2 < 3; ++q2) Gs2.a[p][q2] = dSt.a[p][q2] + dSt.a[q2][p];
    M3<double> dA = mul(mul(Gs2, P.A), Sigma);
    M3<double> dSigma = mul(mul(transpose(P.A), dSt), P.A);
    // A = J W: dJ = dA W^T
    M3<double> dJ = mul(dA, transpose(Wm));
    double du[3] = {0, 0, 0};
    const double u0 = P.u[0], u1 = P.u[1], u2 = P.u[2];
    if (cam.beam == 1) {
        const double L = cam.L_SD;
        const double l = std::sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        du[2] += -(dJ.a[0][0] + dJ.a[1][1]) * L / (u2 * u2);
        du[0] += -dJ.a[0][2] * L / (u2 * u2);
        du[2] += dJ.a[0][2] * 2.0 * L * u0 / (u2 * u2 * u2);
        du[1] += -dJ.a[1][2] * L / (u2 * u2);
        du[2] += dJ.a[1][2] * 2.0 * L * u1 / (u2 * u2 * u2);
        // third row u/l
        const double n[3] = {u0 / l, u1 / l, u2 / l};
        const double g3[3] = {dJ.a[2][0], dJ.a[2][1], dJ.a[2][2]};
        const double nd = n[0] * g3[0] + n[1] * g3[1] + n[2] * g3[2];
        for (int k = 0; k < 3; ++k) du[k] += (g3[k] - n[k] * nd) / l;
        // p^ = L (u0/u2, u1/u2)
        du[0] += d_ph0 * L / u2;
        du[1] += d_ph1 * L / u2;
        du[2] += -(d_ph0 * u0 + d_ph1 * u1) * L / (u2 * u2);
    } else {
        du[0] += d_ph0;
        du[1] += d_ph1;
    }
    // u = W p + t
    for (int k = 0; k < 3; ++k) g.mean[3 * oi + k] += Wm.a[0][k] * du[0] + Wm.a[1][k] * du[1] + Wm.a[2][k] * du[2];
    sigma_backward(dSigma, R, &G.scale[3 * i], qn, qnorm, &g.scale[3 * oi], &g.quat[4 * oi]);
}

// Record gradient of one (pixel, Gaussian) pair with dL/dI = gI.
inline void pair_record_grad(const Proj<double>& P, double dx, double dy, double q, double gI, double out[6]) {
    const double a = P.conic[0], b = P.conic[1], c = P.conic[2];
    const double e = std::exp(-0.5 * q);
    const double dq = -0.5 * gI * P.rhohat * e;
    out[0] = gI * e;
    out[1] = -dq * (2 * a * dx + 2 * b * dy);
    out[2] = -dq * (2 * b * dx + 2 * c * dy);
    out[3] = dq * dx * dx;
    out[4] = dq * 2 * dx * dy;
    out[5] = dq * dy * dy;
}

// band (optional): per parameter, the summed |gradient contribution| of the pairs
// whose q lies within 1e-4 Q of the gate -- the most an FP32 gate decision can move
// that parameter's gradient.
void render_backward(const Params& Pm, const double* views, int V, const Cam& cam, double Q,
                     const double* dimg, Grad g, const Grad* band) {
    const int H = cam.H, Wd = cam.W;
    const ParamsT<double> G = widen<double>(Pm);
    std::vector<double> tm(3), ts(3), tq(4), tr(1);
    for (int v = 0; v < V; ++v) {
        const double* view = views + 12 * v;
        M3<double> Wm;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Wm.a[i][j] = view[3 * i + j];
        const double* dIv = dimg + (int64_t)v * H * Wd;
        for (int64_t i = 0; i < Pm.M; ++i) {
            M3<double> Sigma, R;
            double qn[4], qnorm;
            covariance(&G.scale[3 * i], &G.quat[4 * i], Sigma, R, qn, qnorm);
            Proj<double> P = project_one(&G.mean[3 * i], Sigma, G.rho[i], view, cam);
            if (!P.valid) continue;
            int c0, c1, r0, r1;
            centre_range(P.ph[0], std::sqrt(Q * P.shd[0]), cam.pitch_u, cam.off_u, Wd, c0, c1);
            centre_range(P.ph[1], std::sqrt(Q * P.shd[2]), cam.pitch_v, cam.off_v, H, r0, r1);
            const double a = P.conic[0], b = P.conic[1], c = P.conic[2];
            double drec[6] = {0, 0, 0, 0, 0, 0};
            for (int r = r0; r <= r1; ++r) {
                const double dy = pix_eta(r, cam) - P.ph[1];
                for (int cc = c0; cc <= c1; ++cc) {
                    const double dx = pix_xi(cc, cam) - P.ph[0];
                    const double q = a * dx * dx + 2 * b * dx * dy + c * dy * dy;
                    const double gI = dIv[(int64_t)r * Wd + cc];
                    double pr[6];
                    if (band && std::fabs(q - Q) <= 1e-4 * Q) {
                        pair_record_grad(P, dx, dy, q, gI, pr);
                        std::fill(tm.begin(), tm.end(), 0.0);
                        std::fill(ts.begin(), ts.end(), 0.0);
                        std::fill(tq.begin(), tq.end(), 0.0);
                        tr[0] = 0.0;
                        const Grad tg{tm.data(), ts.data(), tq.data(), tr.data()};
                        chain_record(P, Sigma, R, qn, qnorm, Wm, cam, G, i, pr, tg, 0);
                        for (int k = 0; k < 3; ++k) {
                            band->mean[3 * i + k] += std::fabs(tm[k]);
                            band->scale[3 * i + k] += std::fabs(ts[k]);
                        }
                        for (int k = 0; k < 4; ++k) band->quat[4 * i + k] += std::fabs(tq[k]);
                        band->rho[i] += std::fabs(tr[0]);
                    }
                    if (!(q <= Q)) continue;
                    pair_record_grad(P, dx, dy, q, gI, pr);
                    for (int k = 0; k < 6; ++k) drec[k] += pr[k];
                }
            }
            chain_record(P, Sigma, R, qn, qnorm, Wm, cam, G, i, drec, g, i);
        }
    }
}

// Per (view, Gaussian) record gradient d(rho_hat, p^x, p^y, a, b, c) of the gated
// image sum for dL/dI = dimg (detector units), out[v][i][6]; zeros for records
// that are dropped or touch no gated pixel.
void record_grads(const Params& Pm, const double* views, int V, const Cam& cam, double Q, const double* dimg,
                  double* out) {
    const int H = cam.H, Wd = cam.W;
    const ParamsT<double> G = widen<double>(Pm);
    for (int v = 0; v < V; ++v) {
        const double* view = views + 12 * v;
        const double* dIv = dimg + (int64_t)v * H * Wd;
        for (int64_t i = 0; i < Pm.M; ++i) {
            double* drec = out + ((int64_t)v * Pm.M + i) * 6;
            for (int k = 0; k < 6; ++k) drec[k] = 0.0;
            M3<double> Sigma, R;
            double qn[4], qnorm;
            covariance(&G.scale[3 * i], &G.quat[4 * i], Sigma, R, qn, qnorm);
            Proj<double> P = project_one(&G.mean[3 * i], Sigma, G.rho[i], view, cam);
            if (!P.valid) continue;
            int c0, c1, r0, r1;
            centre_range(P.ph[0], std::sqrt(Q * P.shd[0]), cam.pitch_u, cam.off_u, Wd, c0, c1);
            centre_range(P.ph[1], std::sqrt(Q * P.shd[2]), cam.pitch_v, cam.off_v, H, r0, r1);
            const double a = P.conic[0], b = P.conic[1], c = P.conic[2];
            for (int r = r0; r <= r1; ++r) {
                const double dy = pix_eta(r, cam) - P.ph[1];
                for (int cc = c0; cc <= c1; ++cc) {
                    const double dx = pix_xi(cc, cam) - P.ph[0];
                    const double q = a * dx * dx + 2 * b * dx * dy + c * dy * dy;
                    if (!(q <= Q)) continue;
                    double pr[6];
                    pair_record_grad(P, dx, dy, q, dIv[(int64_t)r * Wd + cc], pr);
                    for (int k = 0; k < 6; ++k) drec[k] += pr[k];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// O1 voxelizer (Eq. 4): V[x] = sum_i rho_i exp(-1/2 (x-p_i)^T Sigma_i^{-1} (x-p_i)) [q <= Q3]
// at voxel centres x = origin + (idx + 1/2) * voxel.  Grid layout [Z][Y][X].

struct GridSpec {
    double origin[3], voxel[3];
    int dims[3];  // X, Y, Z
};

inline void grids_from(const double* gdesc, int G, std::vector<GridSpec>& out) {
    out.resize(G);
    for (int g = 0; g < G; ++g) {
        const double* d = gdesc + 9 * g;
        for (int k = 0; k < 3; ++k) {
            out[g].origin[k] = d[k];
            out[g].voxel[k] = d[3 + k];
            out[g].dims[k] = (int)d[6 + k];
        }
    }
}

template <class T>
int64_t voxelize(const ParamsT<T>& Gp, int64_t M, const std::vector<GridSpec>& grids, double Q3, T* vol,
                 double* band, bool brute) {
    int64_t off = 0, pairs = 0;
    for (const GridSpec& gs : grids) {
        const int X = gs.dims[0], Y = gs.dims[1], Z = gs.dims[2];
        T* Vg = vol + off;
        double* Bg = band ? band + off : nullptr;
        for (int64_t k = 0; k < (int64_t)X * Y * Z; ++k) Vg[k] = 0.0;
        if (Bg)
            for (int64_t k = 0; k < (int64_t)X * Y * Z; ++k) Bg[k] = 0.0;
        for (int64_t i = 0; i < M; ++i) {
            M3<T> Sigma, R;
            T qn[4], qnorm;
            covariance(&Gp.scale[3 * i], &Gp.quat[4 * i], Sigma, R, qn, qnorm);
            M3<T> P = inverse(Sigma);
            const T* p = &Gp.mean[3 * i];
            int lo[3], hi[3];
            for (int k = 0; k < 3; ++k) {
                lo[k] = 0;
                hi[k] = gs.dims[k] - 1;
                if (!brute) {
                    const double e = std::sqrt(Q3 * re(Sigma.a[k][k]));
                    // voxel centre x = origin + (idx + 1/2) voxel; same widened range as pixels
                    const double a = (re(p[k]) - e - gs.origin[k]) / gs.voxel[k] - 0.5;
                    const double b = (re(p[k]) + e - gs.origin[k]) / gs.voxel[k] - 0.5;
                    lo[k] = (int)std::max(-1.0, std::min((double)gs.dims[k], std::ceil(a) - 1.0));
                    hi[k] = (int)std::max(-1.0, std::min((double)gs.dims[k], std::floor(b) + 1.0));
                    lo[k] = std::max(lo[k], 0);
                    hi[k] = std::min(hi[k], gs.dims[k] - 1);
                }
            }
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        const double xc[3] = {gs.origin[0] + (x + 0.5) * gs.voxel[0],
                                              gs.origin[1] + (y + 0.5) * gs.voxel[1],
                                              gs.origin[2] + (z + 0.5) * gs.voxel[2]};
                        T d[3];
                        for (int k = 0; k < 3; ++k) d[k] = xc[k] - p[k];
                        T q = 0.0;
                        for (int j = 0; j < 3; ++j)
                            for (int k = 0; k < 3; ++k) q += d[j] * P.a[j][k] * d[k];
                        const double qr = re(q);
                        const int64_t idx = ((int64_t)z * Y + y) * X + x;
                        if (Bg && std::fabs(qr - Q3) <= 1e-4 * Q3)
                            Bg[idx] += std::fabs(re(Gp.rho[i])) * std::exp(-0.5 * qr);
                        if (!(qr <= Q3)) continue;
                        Vg[idx] += Gp.rho[i] * std::exp(-0.5 * q);
                        ++pairs;
                    }
        }
        off += (int64_t)X * Y * Z;
    }
    return pairs;
}

// O1 voxelizer with each Gaussian's gate held at a second parameter set Gg (see
// render_gated): the voxels with q <= Q3 for Gaussian i of Gg receive
// rho_i exp(-q/2) of Gaussian i of G.
int64_t voxelize_gated(const ParamsT<double>& Gp, const ParamsT<double>& Gg, int64_t M,
                       const std::vector<GridSpec>& grids, double Q3, double* vol) {
    int64_t off = 0, pairs = 0;
    for (const GridSpec& gs : grids) {
        const int X = gs.dims[0], Y = gs.dims[1], Z = gs.dims[2];
        double* Vg = vol + off;
        for (int64_t k = 0; k < (int64_t)X * Y * Z; ++k) Vg[k] = 0.0;
        for (int64_t i = 0; i < M; ++i) {
            M3<double> Sg, Rg, S, R;
            double qg[4], ng, qn[4], nn;
            covariance(&Gg.scale[3 * i], &Gg.quat[4 * i], Sg, Rg, qg, ng);
            covariance(&Gp.scale[3 * i], &Gp.quat[4 * i], S, R, qn, nn);
            const M3<double> Pg = inverse(Sg), P = inverse(S);
            const double* pg = &Gg.mean[3 * i];
            const double* p = &Gp.mean[3 * i];
            int lo[3], hi[3];
            for (int k = 0; k < 3; ++k) {
                const double e = std::sqrt(Q3 * Sg.a[k][k]);
                const double a = (pg[k] - e - gs.origin[k]) / gs.voxel[k] - 0.5;
                const double b = (pg[k] + e - gs.origin[k]) / gs.voxel[k] - 0.5;
                lo[k] = std::max(0, (int)std::max(-1.0, std::min((double)gs.dims[k], std::ceil(a) - 1.0)));
                hi[k] = std::min(gs.dims[k] - 1, (int)std::max(-1.0, std::min((double)gs.dims[k], std::floor(b) + 1.0)));
            }
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        const double xc[3] = {gs.origin[0] + (x + 0.5) * gs.voxel[0],
                                              gs.origin[1] + (y + 0.5) * gs.voxel[1],
                                              gs.origin[2] + (z + 0.5) * gs.voxel[2]};
                        double dg[3], d[3];
                        for (int k = 0; k < 3; ++k) {
                            dg[k] = xc[k] - pg[k];
                            d[k] = xc[k] - p[k];
                        }
                        double qgate = 0.0, q = 0.0;
                        for (int j = 0; j < 3; ++j)
                            for (int k = 0; k < 3; ++k) {
                                qgate += dg[j] * Pg.a[j][k] * dg[k];
                                q += d[j] * P.a[j][k] * d[k];
                            }
                        if (!(qgate <= Q3)) continue;
                        Vg[((int64_t)z * Y + y) * X + x] += Gp.rho[i] * std::exp(-0.5 * q);
                        ++pairs;
                    }
        }
        off += (int64_t)X * Y * Z;
    }
    return pairs;
}

// Chain from (d rho, d p, d P) of one Gaussian (P = Sigma^{-1}) to its parameters.
void vox_chain(const M3<double>& P, const M3<double>& R, const double qn[4], double qnorm, const double* s,
               double drho, const double dp[3], const M3<double>& dP, Grad g, int64_t oi) {
    g.rho[oi] += drho;
    for (int k = 0; k < 3; ++k) g.mean[3 * oi + k] += dp[k];
    // P = Sigma^{-1}: dSigma = -P^T dP P^T
    M3<double> Pt = transpose(P);
    M3<double> dSigma = mul(mul(Pt, dP), Pt);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) dSigma.a[j][k] = -dSigma.a[j][k];
    sigma_backward(dSigma, R, s, qn, qnorm, &g.scale[3 * oi], &g.quat[4 * oi]);
}

void voxelize_backward(const Params& Pm, const std::vector<GridSpec>& grids, double Q3, const double* dvol,
                       Grad g, const Grad* band) {
    const ParamsT<double> Gp = widen<double>(Pm);
    double tm[3], ts[3], tq[4], tr[1];
    int64_t off = 0;
    for (const GridSpec& gs : grids) {
        const int X = gs.dims[0], Y = gs.dims[1], Z = gs.dims[2];
        const double* dV = dvol + off;
        for (int64_t i = 0; i < Pm.M; ++i) {
            M3<double> Sigma, R;
            double qn[4], qnorm;
            covariance(&Gp.scale[3 * i], &Gp.quat[4 * i], Sigma, R, qn, qnorm);
            M3<double> P = inverse(Sigma);
            const double* p = &Gp.mean[3 * i];
            const double rho = Gp.rho[i];
            int lo[3], hi[3];
            for (int k = 0; k < 3; ++k) {
                const double e = std::sqrt(Q3 * Sigma.a[k][k]);
                const double a = (p[k] - e - gs.origin[k]) / gs.voxel[k] - 0.5;
                const double b = (p[k] + e - gs.origin[k]) / gs.voxel[k] - 0.5;
                lo[k] = (int)std::max(-1.0, std::min((double)gs.dims[k], std::ceil(a) - 1.0));
                hi[k] = (int)std::max(-1.0, std::min((double)gs.dims[k], std::floor(b) + 1.0));
                lo[k] = std::max(lo[k], 0);
                hi[k] = std::min(hi[k], gs.dims[k] - 1);
            }
            double drho = 0, dp[3] = {0, 0, 0};
            M3<double> dP{};
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        const double xc[3] = {gs.origin[0] + (x + 0.5) * gs.voxel[0],
                                              gs.origin[1] + (y + 0.5) * gs.voxel[1],
                                              gs.origin[2] + (z + 0.5) * gs.voxel[2]};
                        double d[3];
                        for (int k = 0; k < 3; ++k) d[k] = xc[k] - p[k];
                        double q = 0.0;
                        for (int j = 0; j < 3; ++j)
                            for (int k = 0; k < 3; ++k) q += d[j] * P.a[j][k] * d[k];
                        const bool in_band = band && std::fabs(q - Q3) <= 1e-4 * Q3;
                        if (!(q <= Q3) && !in_band) continue;
                        const double gv = dV[((int64_t)z * Y + y) * X + x];
                        const double e = std::exp(-0.5 * q);
                        // one pair: d rho = g e; q = d^T P d, d = x - p:
                        // dq/dp = -(P + P^T) d, dq/dP_jk = d_j d_k
                        const double dq = -0.5 * gv * rho * e;
                        double pdp[3];
                        M3<double> pdP{};
                        for (int j = 0; j < 3; ++j) {
                            double Pd = 0;
                            for (int k = 0; k < 3; ++k) Pd += (P.a[j][k] + P.a[k][j]) * d[k];
                            pdp[j] = -dq * Pd;
                            for (int k = 0; k < 3; ++k) pdP.a[j][k] = dq * d[j] * d[k];
                        }
                        if (in_band) {
                            std::fill(tm, tm + 3, 0.0);
                            std::fill(ts, ts + 3, 0.0);
                            std::fill(tq, tq + 4, 0.0);
                            tr[0] = 0.0;
                            vox_chain(P, R, qn, qnorm, &Gp.scale[3 * i], gv * e, pdp, pdP, Grad{tm, ts, tq, tr}, 0);
                            for (int k = 0; k < 3; ++k) {
                                band->mean[3 * i + k] += std::fabs(tm[k]);
                                band->scale[3 * i + k] += std::fabs(ts[k]);
                            }
                            for (int k = 0; k < 4; ++k) band->quat[4 * i + k] += std::fabs(tq[k]);
                            band->rho[i] += std::fabs(tr[0]);
                        }
                        if (!(q <= Q3)) continue;
                        drho += gv * e;
                        for (int j = 0; j < 3; ++j) {
                            dp[j] += pdp[j];
                            for (int k = 0; k < 3; ++k) dP.a[j][k] += pdP.a[j][k];
                        }
                    }
            vox_chain(P, R, qn, qnorm, &Gp.scale[3 * i], drho, dp, dP, g, i);
        }
        off += (int64_t)X * Y * Z;
    }
}

// ---------------------------------------------------------------------------
// O2 / O3: one Gaussian along the ray s + t*omega, |omega| = 1, t over R.

struct Ray {
    double s[3], w[3];
};

// The ray of detector pixel (r, c) in view v, in world coordinates.
// cone: from the source (scanner origin) through the pixel centre on the plane u2 = L_SD;
// parallel: along the scanner's third axis through (xi, eta, 0).
Ray pixel_ray(const double* view, const Cam& cam, int r, int c) {
    double Wm[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Wm[i][j] = view[3 * i + j];
        t[i] = view[9 + i];
    }
    const double xi = pix_xi(c, cam), eta = pix_eta(r, cam);
    Ray ray;
    double us[3], ud[3];
    if (cam.beam == 1) {
        us[0] = 0; us[1] = 0; us[2] = 0;
        ud[0] = xi; ud[1] = eta; ud[2] = cam.L_SD;
    } else {
        us[0] = xi; us[1] = eta; us[2] = 0;
        ud[0] = 0; ud[1] = 0; ud[2] = 1;
    }
    // world = W^T (u - t) for points, W^T d for directions (W orthonormal)
    double nrm = std::sqrt(ud[0] * ud[0] + ud[1] * ud[1] + ud[2] * ud[2]);
    for (int k = 0; k < 3; ++k) {
        ray.s[k] = Wm[0][k] * (us[0] - t[0]) + Wm[1][k] * (us[1] - t[1]) + Wm[2][k] * (us[2] - t[2]);
        ray.w[k] = (Wm[0][k] * ud[0] + Wm[1][k] * ud[1] + Wm[2][k] * ud[2]) / nrm;
    }
    return ray;
}

// closed form: rho sqrt(2 pi / a) exp(-1/2 (c - b^2/a)), a = w^T P w, b = w^T P (p - s), c = (p-s)^T P (p-s)
double ray_integral(const double* p, const M3<double>& P, double rho, const Ray& ray) {
    double d[3], Pw[3], Pd[3];
    for (int k = 0; k < 3; ++k) d[k] = p[k] - ray.s[k];
    for (int j = 0; j < 3; ++j) {
        Pw[j] = P.a[j][0] * ray.w[0] + P.a[j][1] * ray.w[1] + P.a[j][2] * ray.w[2];
        Pd[j] = P.a[j][0] * d[0] + P.a[j][1] * d[1] + P.a[j][2] * d[2];
    }
    const double a = ray.w[0] * Pw[0] + ray.w[1] * Pw[1] + ray.w[2] * Pw[2];
    const double b = ray.w[0] * Pd[0] + ray.w[1] * Pd[1] + ray.w[2] * Pd[2];
    const double c = d[0] * Pd[0] + d[1] * Pd[1] + d[2] * Pd[2];
    return rho * std::sqrt(2.0 * M_PI / a) * std::exp(-0.5 * (c - b * b / a));
}

// trapezoid rule over [t* - 12 sr, t* + 12 sr] with step sr/8, t* = b/a, sr = a^{-1/2}
double ray_quadrature(const double* p, const M3<double>& P, double rho, const Ray& ray) {
    double d[3], Pw[3], Pd[3];
    for (int k = 0; k < 3; ++k) d[k] = p[k] - ray.s[k];
    for (int j = 0; j < 3; ++j) {
        Pw[j] = P.a[j][0] * ray.w[0] + P.a[j][1] * ray.w[1] + P.a[j][2] * ray.w[2];
        Pd[j] = P.a[j][0] * d[0] + P.a[j][1] * d[1] + P.a[j][2] * d[2];
    }
    const double a = ray.w[0] * Pw[0] + ray.w[1] * Pw[1] + ray.w[2] * Pw[2];
    const double b = ray.w[0] * Pd[0] + ray.w[1] * Pd[1] + ray.w[2] * Pd[2];
    const double ts = b / a, sr = 1.0 / std::sqrt(a), h = sr / 8.0;
    double sum = 0.0;
    for (int k = -96; k <= 96; ++k) {
        const double t = ts + k * h;
        double e[3];
        for (int j = 0; j < 3; ++j) e[j] = ray.s[j] + t * ray.w[j] - p[j];
        double q = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) q += e[i] * P.a[i][j] * e[j];
        const double wgt = (k == -96 || k == 96) ? 0.5 : 1.0;
        sum += wgt * rho * std::exp(-0.5 * q);
    }
    return sum * h;
}

Cam make_cam(const double* c) {
    Cam cam;
    cam.beam = (int)c[0];
    cam.H = (int)c[1];
    cam.W = (int)c[2];
    cam.L_SD = c[3];
    cam.pitch_u = c[4];
    cam.pitch_v = c[5];
    cam.off_u = c[6];
    cam.off_v = c[7];
    cam.near_plane = c[8];
    cam.jmode = (int)c[9];
    cam.biased = (int)c[10];
    cam.dilation = c[11];
    return cam;
}

// ---------------------------------------------------------------------------
// R32: the stated FP32 op sequence for p^, Sigma^ and the tile bound.  Every
// operation below is one IEEE single-precision +, -, *, / or sqrt, evaluated in
// the written order, no fused multiply-add (built with -ffp-contract=off).

struct F32Out {
    float ph[2], sh[3], u2, det;
    int valid;
    int pix[4];   // c_lo, c_hi, r_lo, r_hi (pixel centres), inclusive
    int tile[4];  // tx_lo, tx_hi, ty_lo, ty_hi, inclusive
};

static inline float f_ceil_clamped(float x, int n) {
    // ceil(x) clamped into [-1, n] before the integer conversion
    if (!(x > -1.0f)) return -1.0f;
    if (x > (float)n) return (float)n;
    return std::ceil(x);
}
static inline float f_floor_clamped(float x, int n) {
    if (!(x > -1.0f)) return -1.0f;
    if (x > (float)n) return (float)n;
    return std::floor(x);
}

F32Out project_f32(const float* p, const float* s, const float* q, const float* view, int beam, float L_SD,
                   int H, int Wd, float pitch_u, float pitch_v, float off_u, float off_v, float near_plane,
                   float Q, int TW, int TH, float dilation) {
    F32Out o{};
    o.valid = 0;
    const float w0 = q[0], x0 = q[1], y0 = q[2], z0 = q[3];
    const float n2 = ((w0 * w0 + x0 * x0) + y0 * y0) + z0 * z0;
    const float n = std::sqrt(n2);
    const float w = w0 / n, x = x0 / n, y = y0 / n, z = z0 / n;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    float Mm[3][3];  // M = R S
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) Mm[j][k] = R[j][k] * s[k];
    float u[3];
    for (int j = 0; j < 3; ++j)
        u[j] = ((view[3 * j + 0] * p[0] + view[3 * j + 1] * p[1]) + view[3 * j + 2] * p[2]) + view[9 + j];
    o.u2 = u[2];
    float T[2][3];  // first two rows of J W
    if (beam == 1) {
        if (!(u[2] > near_plane)) return o;
        const float f = L_SD / u[2];
        const float j02 = -((f * u[0]) / u[2]);
        const float j12 = -((f * u[1]) / u[2]);
        o.ph[0] = f * u[0];
        o.ph[1] = f * u[1];
        for (int k = 0; k < 3; ++k) {
            T[0][k] = f * view[0 * 3 + k] + j02 * view[2 * 3 + k];
            T[1][k] = f * view[1 * 3 + k] + j12 * view[2 * 3 + k];
        }
    } else {
        o.ph[0] = u[0];
        o.ph[1] = u[1];
        for (int k = 0; k < 3; ++k) {
            T[0][k] = view[0 * 3 + k];
            T[1][k] = view[1 * 3 + k];
        }
    }
    // N = T M (2x3); Sigma^ = N N^T; |Sigma^| by Cauchy-Binet as a sum of squared 2x2 minors
    float N[2][3];
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k) N[a][k] = (T[a][0] * Mm[0][k] + T[a][1] * Mm[1][k]) + T[a][2] * Mm[2][k];
    const float al = (N[0][0] * N[0][0] + N[0][1] * N[0][1]) + N[0][2] * N[0][2];
    const float be = (N[0][0] * N[1][0] + N[0][1] * N[1][1]) + N[0][2] * N[1][2];
    const float ga = (N[1][0] * N[1][0] + N[1][1] * N[1][1]) + N[1][2] * N[1][2];
    const float m01 = N[0][0] * N[1][1] - N[0][1] * N[1][0];
    const float m02 = N[0][0] * N[1][2] - N[0][2] * N[1][0];
    const float m12 = N[0][1] * N[1][2] - N[0][2] * N[1][1];
    o.sh[0] = al;
    o.sh[1] = be;
    o.sh[2] = ga;
    o.det = (m01 * m01 + m02 * m02) + m12 * m12;
    if (dilation > 0.0f) {
        // footprint Sigma^ + diag(dx, dy), dx = dilation pitch_u^2, dy = dilation pitch_v^2;
        // its determinant expanded as |Sigma^| + (dy alpha + dx gamma) + dx dy
        const float dx = (dilation * pitch_u) * pitch_u, dy = (dilation * pitch_v) * pitch_v;
        o.det = (o.det + (dy * al + dx * ga)) + dx * dy;
        o.sh[0] = al + dx;
        o.sh[2] = ga + dy;
    }
    if (!(o.det > 0.0f)) return o;
    const float ex = std::sqrt(Q * o.sh[0]), ey = std::sqrt(Q * o.sh[2]);
    const float hw = 0.5f * (float)Wd - 0.5f, hh = 0.5f * (float)H - 0.5f;
    const float cx = (o.ph[0] - off_u) / pitch_u + hw;
    const float cy = (o.ph[1] - off_v) / pitch_v + hh;
    const float rx = ex / pitch_u, ry = ey / pitch_v;
    const int c_lo = std::max(0, (int)f_ceil_clamped(cx - rx, Wd));
    const int c_hi = std::min(Wd - 1, (int)f_floor_clamped(cx + rx, Wd));
    const int r_lo = std::max(0, (int)f_ceil_clamped(cy - ry, H));
    const int r_hi = std::min(H - 1, (int)f_floor_clamped(cy + ry, H));
    if (c_lo > c_hi || r_lo > r_hi) return o;
    o.valid = 1;
    o.pix[0] = c_lo; o.pix[1] = c_hi; o.pix[2] = r_lo; o.pix[3] = r_hi;
    o.tile[0] = c_lo / TW; o.tile[1] = c_hi / TW; o.tile[2] = r_lo / TH; o.tile[3] = r_hi / TH;
    return o;
}

// FP32 brick bound for the voxelizer: Sigma_kk by the same op sequence as above,
// e_k = sqrt(Q3 Sigma_kk), centre c_k = (p_k - origin_k)/voxel_k - 1/2, r_k = e_k/voxel_k.
int brick_bound_f32(const float* p, const float* s, const float* q, const float* origin, const float* voxel,
                    const int* dims, float Q3, int B, int* out /* lo[3], hi[3] voxels, then bricks lo[3], hi[3] */) {
    const float w0 = q[0], x0 = q[1], y0 = q[2], z0 = q[3];
    const float n2 = ((w0 * w0 + x0 * x0) + y0 * y0) + z0 * z0;
    const float n = std::sqrt(n2);
    const float w = w0 / n, x = x0 / n, y = y0 / n, z = z0 / n;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
    float Mm[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) Mm[j][k] = R[j][k] * s[k];
    for (int k = 0; k < 3; ++k) {
        const float skk = (Mm[k][0] * Mm[k][0] + Mm[k][1] * Mm[k][1]) + Mm[k][2] * Mm[k][2];
        const float e = std::sqrt(Q3 * skk);
        const float c = (p[k] - origin[k]) / voxel[k] - 0.5f;
        const float r = e / voxel[k];
        const int lo = std::max(0, (int)f_ceil_clamped(c - r, dims[k]));
        const int hi = std::min(dims[k] - 1, (int)f_floor_clamped(c + r, dims[k]));
        if (lo > hi) return 0;
        out[k] = lo;
        out[3 + k] = hi;
        out[6 + k] = lo / B;
        out[9 + k] = hi / B;
    }
    return 1;
}

}  // namespace

// ===========================================================================
// C entry points for the Python test harness (ctypes).

extern "C" {

// cam: [beam, H, W, L_SD, pitch_u, pitch_v, off_u, off_v, near_plane, jmode, biased, dilation]
int64_t orc_render(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                   const double* views, int V, const double* camv, double Q, int brute, double* img, double* band) {
    const Params P{M, mean, scale, quat, rho};
    const Cam cam = make_cam(camv);
    ParamsT<double> G = widen<double>(P);
    return render<double>(G, M, views, V, cam, Q, img, band, brute != 0);
}

// render_gated: values from (mean, scale, quat, rho), gates from the g* set.
int64_t orc_render_gated(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                         const double* gmean, const double* gscale, const double* gquat, const double* grho,
                         const double* views, int V, const double* camv, double Q, double* img) {
    const ParamsT<double> G = widen<double>(Params{M, mean, scale, quat, rho});
    const ParamsT<double> Gg = widen<double>(Params{M, gmean, gscale, gquat, grho});
    return render_gated(G, Gg, M, views, V, make_cam(camv), Q, img);
}

// voxelize_gated: values from (mean, scale, quat, rho), gates from the g* set.
int64_t orc_voxelize_gated(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                           const double* gmean, const double* gscale, const double* gquat, const double* grho,
                           const double* gdesc, int G, double Q3, double* vol) {
    std::vector<GridSpec> grids;
    grids_from(gdesc, G, grids);
    const ParamsT<double> Gp = widen<double>(Params{M, mean, scale, quat, rho});
    const ParamsT<double> Gg = widen<double>(Params{M, gmean, gscale, gquat, grho});
    return voxelize_gated(Gp, Gg, M, grids, Q3, vol);
}

// Per (Gaussian, view) projection quantities in FP64: out[v][i][12] =
// valid, p^x, p^y, alpha, beta, gamma, |Sigma~|, |Sigma^|, mu, rho_hat, u2, |u|
void orc_project(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                 const double* views, int V, const double* camv, double* out) {
    const Cam cam = make_cam(camv);
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < M; ++i) {
            M3<double> Sigma, R;
            double qn[4], qnorm;
            covariance(&scale[3 * i], &quat[4 * i], Sigma, R, qn, qnorm);
            Proj<double> P = project_one(&mean[3 * i], Sigma, rho[i], views + 12 * v, cam);
            double* o = out + ((int64_t)v * M + i) * 12;
            o[0] = P.valid ? 1.0 : 0.0;
            o[1] = P.ph[0]; o[2] = P.ph[1];
            o[3] = P.sh[0]; o[4] = P.sh[1]; o[5] = P.sh[2];
            o[6] = P.d3; o[7] = P.d2; o[8] = P.mu; o[9] = P.rhohat;
            o[10] = P.u[2];
            o[11] = std::sqrt(P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]);
        }
}

// Mean over the views of the integration-bias factor mu = sqrt(2 pi |Sigma~| / |Sigma^|)
// of each Gaussian (Eq. 7), counting only the views in which it projects (cone beam:
// u2 > near plane); 0 where it projects in none.  mu_mean[i] for Gaussian i.
void orc_mean_mu(int64_t M, const double* mean, const double* scale, const double* quat, const double* views,
                 int V, const double* camv, double* mu_mean) {
    const Cam cam = make_cam(camv);
    for (int64_t i = 0; i < M; ++i) {
        M3<double> Sigma, R;
        double qn[4], qnorm;
        covariance(&scale[3 * i], &quat[4 * i], Sigma, R, qn, qnorm);
        double sum = 0.0;
        int n = 0;
        for (int v = 0; v < V; ++v) {
            Proj<double> P = project_one(&mean[3 * i], Sigma, 1.0, views + 12 * v, cam);
            if (!P.valid) continue;
            sum += P.mu;
            ++n;
        }
        mu_mean[i] = n ? sum / n : 0.0;
    }
}

void orc_record_grads(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                      const double* views, int V, const double* camv, double Q, const double* dimg, double* out) {
    record_grads(Params{M, mean, scale, quat, rho}, views, V, make_cam(camv), Q, dimg, out);
}

// Complex-step derivative of the whole image with respect to one parameter:
// kind 0 mean, 1 scale, 2 quat, 3 rho; element index i, component comp.
// out[v][r][c] = Im(I(theta + i h e)) / h.
void orc_render_cs(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                   const double* views, int V, const double* camv, double Q, int kind, int64_t i, int comp,
                   double h, double* out) {
    const Params P{M, mean, scale, quat, rho};
    const Cam cam = make_cam(camv);
    ParamsT<cd> G = widen<cd>(P);
    cd* tgt = nullptr;
    if (kind == 0) tgt = &G.mean[3 * i + comp];
    if (kind == 1) tgt = &G.scale[3 * i + comp];
    if (kind == 2) tgt = &G.quat[4 * i + comp];
    if (kind == 3) tgt = &G.rho[i];
    *tgt += cd(0.0, h);
    std::vector<cd> img((size_t)V * cam.H * cam.W);
    render<cd>(G, M, views, V, cam, Q, img.data(), nullptr, false);
    for (size_t k = 0; k < img.size(); ++k) out[k] = img[k].imag() / h;
}

// band_* may be NULL (no gate-band bound wanted).
void orc_render_backward(int64_t M, const double* mean, const double* scale, const double* quat,
                         const double* rho, const double* views, int V, const double* camv, double Q,
                         const double* dimg, double* dmean, double* dscale, double* dquat, double* drho,
                         double* band_mean, double* band_scale, double* band_quat, double* band_rho) {
    const Params P{M, mean, scale, quat, rho};
    const Grad band{band_mean, band_scale, band_quat, band_rho};
    render_backward(P, views, V, make_cam(camv), Q, dimg, Grad{dmean, dscale, dquat, drho},
                    band_mean ? &band : nullptr);
}

// grids: [G][9] = origin(3), voxel(3), dims(3: X, Y, Z); volumes concatenated.
int64_t orc_voxelize(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                     const double* gdesc, int G, double Q3, int brute, double* vol, double* band) {
    const Params P{M, mean, scale, quat, rho};
    std::vector<GridSpec> grids;
    grids_from(gdesc, G, grids);
    ParamsT<double> Gp = widen<double>(P);
    return voxelize<double>(Gp, M, grids, Q3, vol, band, brute != 0);
}

void orc_voxelize_cs(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                     const double* gdesc, int G, double Q3, int kind, int64_t i, int comp, double h, double* out) {
    const Params P{M, mean, scale, quat, rho};
    std::vector<GridSpec> grids;
    grids_from(gdesc, G, grids);
    ParamsT<cd> Gp = widen<cd>(P);
    cd* tgt = nullptr;
    if (kind == 0) tgt = &Gp.mean[3 * i + comp];
    if (kind == 1) tgt = &Gp.scale[3 * i + comp];
    if (kind == 2) tgt = &Gp.quat[4 * i + comp];
    if (kind == 3) tgt = &Gp.rho[i];
    *tgt += cd(0.0, h);
    int64_t n = 0;
    for (const GridSpec& g : grids) n += (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
    std::vector<cd> vol((size_t)n);
    voxelize<cd>(Gp, M, grids, Q3, vol.data(), nullptr, false);
    for (int64_t k = 0; k < n; ++k) out[k] = vol[k].imag() / h;
}

// band_* may be NULL (no gate-band bound wanted).
void orc_voxelize_backward(int64_t M, const double* mean, const double* scale, const double* quat,
                           const double* rho, const double* gdesc, int G, double Q3, const double* dvol,
                           double* dmean, double* dscale, double* dquat, double* drho, double* band_mean,
                           double* band_scale, double* band_quat, double* band_rho) {
    const Params P{M, mean, scale, quat, rho};
    std::vector<GridSpec> grids;
    grids_from(gdesc, G, grids);
    const Grad band{band_mean, band_scale, band_quat, band_rho};
    voxelize_backward(P, grids, Q3, dvol, Grad{dmean, dscale, dquat, drho}, band_mean ? &band : nullptr);
}

// O2 over a detector: exact, untruncated, all pixels x all Gaussians.
void orc_render_exact(int64_t M, const double* mean, const double* scale, const double* quat, const double* rho,
                      const double* views, int V, const double* camv, double* img) {
    const Cam cam = make_cam(camv);
    std::vector<M3<double>> Pinv((size_t)M);
    for (int64_t i = 0; i < M; ++i) {
        M3<double> Sigma, R;
        double qn[4], qnorm;
        covariance(&scale[3 * i], &quat[4 * i], Sigma, R, qn, qnorm);
        Pinv[i] = inverse(Sigma);
    }
    for (int v = 0; v < V; ++v)
        for (int r = 0; r < cam.H; ++r)
            for (int c = 0; c < cam.W; ++c) {
                const Ray ray = pixel_ray(views + 12 * v, cam, r, c);
                double s = 0;
                for (int64_t i = 0; i < M; ++i) s += ray_integral(&mean[3 * i], Pinv[i], rho[i], ray);
                img[((int64_t)v * cam.H + r) * cam.W + c] = s;
            }
}

// O2 and O3 for one Gaussian and one arbitrary ray (s, omega normalised here).
void orc_ray_pair(const double* mean, const double* scale, const double* quat, double rho, const double* s,
                  const double* w, double* out2) {
    M3<double> Sigma, R;
    double qn[4], qnorm;
    covariance(scale, quat, Sigma, R, qn, qnorm);
    M3<double> P = inverse(Sigma);
    Ray ray;
    const double n = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int k = 0; k < 3; ++k) {
        ray.s[k] = s[k];
        ray.w[k] = w[k] / n;
    }
    out2[0] = ray_integral(mean, P, rho, ray);
    out2[1] = ray_quadrature(mean, P, rho, ray);
}

// The world ray of one pixel: out = s(3), omega(3).
void orc_pixel_ray(const double* view, const double* camv, int r, int c, double* out) {
    const Ray ray = pixel_ray(view, make_cam(camv), r, c);
    for (int k = 0; k < 3; ++k) {
        out[k] = ray.s[k];
        out[3 + k] = ray.w[k];
    }
}

// R32 projection + tile bounds for all (view, Gaussian) records, record index v*M + i.
// camf: [beam, H, W, L_SD, pitch_u, pitch_v, off_u, off_v, near_plane, dilation] as float.
// out_f[rec][6] = p^x, p^y, alpha, beta, gamma, det ; out_i[rec][9] = valid, pix(4), tile(4)
void orc_project_f32(int64_t M, const float* mean, const float* scale, const float* quat, const float* views,
                     int V, const float* camf, float Q, int TW, int TH, float* out_f, int32_t* out_i) {
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < M; ++i) {
            F32Out o = project_f32(&mean[3 * i], &scale[3 * i], &quat[4 * i], views + 12 * v, (int)camf[0], camf[3],
                                   (int)camf[1], (int)camf[2], camf[4], camf[5], camf[6], camf[7], camf[8], Q, TW,
                                   TH, camf[9]);
            const int64_t rec = (int64_t)v * M + i;
            float* f = out_f + rec * 6;
            f[0] = o.ph[0]; f[1] = o.ph[1]; f[2] = o.sh[0]; f[3] = o.sh[1]; f[4] = o.sh[2]; f[5] = o.det;
            int32_t* n = out_i + rec * 9;
            n[0] = o.valid;
            for (int k = 0; k < 4; ++k) {
                n[1 + k] = o.valid ? o.pix[k] : 0;
                n[5 + k] = o.valid ? o.tile[k] : 0;
            }
        }
}

// R32 brick bounds: gdescf [G][9] as float (origin, voxel, dims). out[g][i][13] = valid, vox lo(3), hi(3),
// brick lo(3), hi(3)
void orc_brick_bounds_f32(int64_t M, const float* mean, const float* scale, const float* quat, const float* gdescf,
                          int G, float Q3, int B, int32_t* out) {
    for (int g = 0; g < G; ++g) {
        const float* d = gdescf + 9 * g;
        const int dims[3] = {(int)d[6], (int)d[7], (int)d[8]};
        for (int64_t i = 0; i < M; ++i) {
            int32_t* o = out + ((int64_t)g * M + i) * 13;
            int tmp[12];
            const int ok = brick_bound_f32(&mean[3 * i], &scale[3 * i], &quat[4 * i], d, d + 3, dims, Q3, B, tmp);
            o[0] = ok;
            for (int k = 0; k < 12; ++k) o[1 + k] = ok ? tmp[k] : 0;
        }
    }
}

}  // extern "C"
