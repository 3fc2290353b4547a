"""ctypes binding of the FP64 C++ oracle (r2g_oracle.cpp).  Test infrastructure only.

Builds ``liboracle.so`` next to the source with g++ (``-ffp-contract=off`` so the
FP32 replica keeps its stated operation order) the first time it is needed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "r2g_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            i64, i32, dbl, flt = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float
            L.orc_render.restype = i64
            L.orc_render.argtypes = [i64, _D, _D, _D, _D, _D, i32, _D, dbl, i32, _D, _D]
            L.orc_render_gated.restype = i64
            L.orc_render_gated.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, _D, _D, i32, _D, dbl, _D]
            L.orc_voxelize_gated.restype = i64
            L.orc_voxelize_gated.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, _D, _D, i32, dbl, _D]
            L.orc_project.restype = None
            L.orc_project.argtypes = [i64, _D, _D, _D, _D, _D, i32, _D, _D]
            L.orc_render_cs.restype = None
            L.orc_render_cs.argtypes = [i64, _D, _D, _D, _D, _D, i32, _D, dbl, i32, i64, i32, dbl, _D]
            L.orc_render_backward.restype = None
            L.orc_render_backward.argtypes = [i64, _D, _D, _D, _D, _D, i32, _D, dbl, _D, _D, _D, _D, _D, _D, _D, _D,
                                              _D]
            L.orc_voxelize.restype = i64
            L.orc_voxelize.argtypes = [i64, _D, _D, _D, _D, _D, i32, dbl, i32, _D, _D]
            L.orc_voxelize_cs.restype = None
            L.orc_voxelize_cs.argtypes = [i64, _D, _D, _D, _D, _D, i32, dbl, i32, i64, i32, dbl, _D]
            L.orc_voxelize_backward.restype = None
            L.orc_voxelize_backward.argtypes = [i64, _D, _D, _D, _D, _D, i32, dbl, _D, _D, _D, _D, _D, _D, _D, _D,
                                                _D]
            L.orc_record_grads.restype = None
            L.orc_record_grads.argtypes = [i64, _D, _D, _D, _D, _D, i32, _D, dbl, _D, _D]
            L.orc_mean_mu.restype = None
            L.orc_mean_mu.argtypes = [i64, _D, _D, _D, _D, i32, _D, _D]
            L.orc_render_exact.restype = None
            L.orc_render_exact.argtypes = [i64, _D, _D, _D, _D, _D, i32, _D, _D]
            L.orc_ray_pair.restype = None
            L.orc_ray_pair.argtypes = [_D, _D, _D, dbl, _D, _D, _D]
            L.orc_pixel_ray.restype = None
            L.orc_pixel_ray.argtypes = [_D, _D, i32, i32, _D]
            L.orc_project_f32.restype = None
            L.orc_project_f32.argtypes = [i64, _F, _F, _F, _F, i32, _F, flt, i32, i32, _F, _I]
            L.orc_brick_bounds_f32.restype = None
            L.orc_brick_bounds_f32.argtypes = [i64, _F, _F, _F, _F, i32, flt, i32, _I]
            _lib = L
    return _lib


def _camv(cam, jmode: int = 0, biased: bool = False, dilation: float = 0.0) -> np.ndarray:
    """Camera vector for the C entry points; jmode 1 plants the depth-row Jacobian
    (used only by the test that pins the EWA reading); biased selects the X-3DGS
    amplitude rho_hat = rho in place of Eq. 7's mu rho; dilation (pixels^2, 0 = none)
    adds dilation * pitch^2 to the diagonal of the footprint evaluated at the pixels
    (3DGS's low-pass filter), leaving mu on the undilated Sigma^."""
    return np.concatenate([np.asarray(cam.as_vector(), dtype=np.float64),
                           [float(jmode), float(bool(biased)), float(dilation)]])


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _f(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _p(a, t=_D):
    return a.ctypes.data_as(t)


class _G:
    """The four parameter arrays widened to float64 (kept alive for ctypes)."""

    def __init__(self, G):
        self.M = int(np.asarray(G.mean).shape[0])
        self.mean, self.scale, self.quat, self.rho = _d(G.mean), _d(G.scale), _d(G.quat), _d(G.rho)

    def ptrs(self):
        return _p(self.mean), _p(self.scale), _p(self.quat), _p(self.rho)


# ----------------------------------------------------------------------------- O1 rasterizer


def render(G, views, cam, Q=9.0, brute=False, want_band=False, jmode=0, biased=False, dilation=0.0):
    """O1 image [V, H, W] (float64), the number of gated (pixel, Gaussian) pairs and,
    if asked, the per-pixel gate-band magnitude."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam, jmode, biased, dilation)
    V = views.shape[0]
    img = np.zeros((V, cam.H, cam.W))
    band = np.zeros((V, cam.H, cam.W)) if want_band else None
    pairs = lib().orc_render(g.M, *g.ptrs(), _p(views), V, _p(cv), float(Q), int(brute), _p(img),
                             _p(band) if band is not None else None)
    return (img, int(pairs), band) if want_band else (img, int(pairs))


def render_gated(G, Ggate, views, cam, Q=9.0):
    """O1 image [V, H, W] of G with every Gaussian's gate (box and q <= Q) taken from
    the same Gaussian of Ggate; equals render(G) when Ggate is G.  Central
    differences of it hold the gate membership fixed."""
    g, gg = _G(G), _G(Ggate)
    assert g.M == gg.M
    views = _d(views)
    cv = _camv(cam)
    img = np.zeros((views.shape[0], cam.H, cam.W))
    lib().orc_render_gated(g.M, *g.ptrs(), *gg.ptrs(), _p(views), views.shape[0], _p(cv), float(Q), _p(img))
    return img


def voxelize_gated(G, Ggate, gdescs, Q3=11.345):
    """O1 volumes (grids concatenated) of G with every Gaussian's gate taken from the
    same Gaussian of Ggate; equals voxelize(G) when Ggate is G."""
    g, gg = _G(G), _G(Ggate)
    assert g.M == gg.M
    gd, G_, n = _grids(gdescs)
    vol = np.zeros(n)
    lib().orc_voxelize_gated(g.M, *g.ptrs(), *gg.ptrs(), _p(gd), G_, float(Q3), _p(vol))
    return vol


def project(G, views, cam, jmode=0, biased=False):
    """FP64 per-(view, Gaussian) quantities [V, M, 12]: valid, p^(2), Sigma^(alpha, beta,
    gamma), |Sigma~|, |Sigma^|, mu, rho_hat, u2, |u|."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam, jmode, biased)
    out = np.zeros((views.shape[0], g.M, 12))
    lib().orc_project(g.M, *g.ptrs(), _p(views), views.shape[0], _p(cv), _p(out))
    return out


def render_cs(G, views, cam, Q, kind, i, comp, h=1e-20, biased=False, dilation=0.0):
    """Complex-step derivative of the image wrt one parameter (kind 0 mean, 1 scale,
    2 quat, 3 rho)."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam, 0, biased, dilation)
    out = np.zeros((views.shape[0], cam.H, cam.W))
    lib().orc_render_cs(g.M, *g.ptrs(), _p(views), views.shape[0], _p(cv), float(Q), kind, i, comp, h, _p(out))
    return out


def _grad_arrays(M):
    return np.zeros((M, 3)), np.zeros((M, 3)), np.zeros((M, 4)), np.zeros(M)


def render_backward(G, views, cam, dimg, Q=9.0, want_band=False, biased=False, dilation=0.0):
    """Hand adjoint: (dmean, dscale, dquat, drho) in float64; with want_band also the
    per-parameter gate-band bound (summed |contribution| of pairs with |q - Q| <= 1e-4 Q)."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam, 0, biased, dilation)
    dimg = _d(dimg)
    out = _grad_arrays(g.M)
    band = _grad_arrays(g.M) if want_band else (None,) * 4
    lib().orc_render_backward(g.M, *g.ptrs(), _p(views), views.shape[0], _p(cv), float(Q), _p(dimg),
                              *(_p(a) for a in out), *((_p(a) if a is not None else None) for a in band))
    return (out, band) if want_band else out


def record_grads(G, views, cam, dimg, Q=9.0, biased=False, dilation=0.0):
    """Per (view, Gaussian) record gradient d(rho_hat, p^x, p^y, a, b, c) of the gated
    image for dL/dI = dimg, [V, M, 6] float64 (p^ in detector units)."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam, 0, biased, dilation)
    dimg = _d(dimg)
    out = np.zeros((views.shape[0], g.M, 6))
    lib().orc_record_grads(g.M, *g.ptrs(), _p(views), views.shape[0], _p(cv), float(Q), _p(dimg), _p(out))
    return out


def mean_mu(G, views, cam):
    """Eq. 7's factor mu of each Gaussian averaged over the views in which it
    projects (0 where it projects in none): [M] float64."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam)
    out = np.zeros(g.M)
    lib().orc_mean_mu(g.M, _p(g.mean), _p(g.scale), _p(g.quat), _p(views), views.shape[0], _p(cv), _p(out))
    return out


def render_exact(G, views, cam):
    """O2: exact, untruncated line integrals for every pixel (all Gaussians)."""
    g = _G(G)
    views = _d(views)
    cv = _camv(cam)
    img = np.zeros((views.shape[0], cam.H, cam.W))
    lib().orc_render_exact(g.M, *g.ptrs(), _p(views), views.shape[0], _p(cv), _p(img))
    return img


def ray_pair(mean, scale, quat, rho, s, w):
    """(O2 closed form, O3 quadrature) for one Gaussian and one ray."""
    out = np.zeros(2)
    m, sc, q, s_, w_ = _d(mean), _d(scale), _d(quat), _d(s), _d(w)
    lib().orc_ray_pair(_p(m), _p(sc), _p(q), float(rho), _p(s_), _p(w_), _p(out))
    return out[0], out[1]


def pixel_ray(view, cam, r, c):
    out = np.zeros(6)
    v = _d(view)
    cv = _camv(cam)
    lib().orc_pixel_ray(_p(v), _p(cv), r, c, _p(out))
    return out[:3], out[3:]


# ----------------------------------------------------------------------------- O1 voxelizer


def _grids(gdescs):
    g = _d(np.atleast_2d(gdescs))
    return g, g.shape[0], int(sum(int(d[6] * d[7] * d[8]) for d in g))


def voxelize(G, gdescs, Q3=11.345, brute=False, want_band=False):
    """O1 volumes, concatenated [sum of X*Y*Z] in [Z][Y][X] order per grid."""
    g = _G(G)
    gd, ng, n = _grids(gdescs)
    vol = np.zeros(n)
    band = np.zeros(n) if want_band else None
    pairs = lib().orc_voxelize(g.M, *g.ptrs(), _p(gd), ng, float(Q3), int(brute), _p(vol),
                               _p(band) if band is not None else None)
    return (vol, int(pairs), band) if want_band else (vol, int(pairs))


def voxelize_cs(G, gdescs, Q3, kind, i, comp, h=1e-20):
    g = _G(G)
    gd, ng, n = _grids(gdescs)
    out = np.zeros(n)
    lib().orc_voxelize_cs(g.M, *g.ptrs(), _p(gd), ng, float(Q3), kind, i, comp, h, _p(out))
    return out


def voxelize_backward(G, gdescs, dvol, Q3=11.345, want_band=False):
    g = _G(G)
    gd, ng, n = _grids(gdescs)
    dvol = _d(dvol).ravel()
    assert dvol.size == n
    out = _grad_arrays(g.M)
    band = _grad_arrays(g.M) if want_band else (None,) * 4
    lib().orc_voxelize_backward(g.M, *g.ptrs(), _p(gd), ng, float(Q3), _p(dvol), *(_p(a) for a in out),
                                *((_p(a) if a is not None else None) for a in band))
    return (out, band) if want_band else out


# ----------------------------------------------------------------------------- R32 replica


def project_f32(G, views, cam, Q=9.0, tile=(16, 16), dilation=0.0):
    """FP32 replica of the stated projection and tile-bound sequence.
    Returns (f [V, M, 6] = p^x, p^y, alpha, beta, gamma, det;
             i [V, M, 9] = valid, pixel c_lo, c_hi, r_lo, r_hi, tile x_lo, x_hi, y_lo, y_hi)."""
    M = int(np.asarray(G.mean).shape[0])
    mean, scale, quat = _f(G.mean), _f(G.scale), _f(G.quat)
    views = _f(views)
    cf = _f(np.concatenate([np.asarray(cam.as_vector(), np.float64), [float(dilation)]]))
    V = views.shape[0]
    out_f = np.zeros((V, M, 6), dtype=np.float32)
    out_i = np.zeros((V, M, 9), dtype=np.int32)
    lib().orc_project_f32(M, _p(mean, _F), _p(scale, _F), _p(quat, _F), _p(views, _F), V, _p(cf, _F),
                          float(Q), int(tile[0]), int(tile[1]), _p(out_f, _F), _p(out_i, _I))
    return out_f, out_i


def tile_lists_f32(G, views, cam, Q=9.0, tile=(16, 16), dilation=0.0):
    """Per-tile Gaussian lists from the R32 bounds: dict tile_key -> sorted array of
    Gaussian ids, tile_key = (v * tiles_y + ty) * tiles_x + tx."""
    _, oi = project_f32(G, views, cam, Q, tile, dilation)
    TW, TH = tile
    tx_n = (cam.W + TW - 1) // TW
    ty_n = (cam.H + TH - 1) // TH
    lists: dict[int, list[int]] = {}
    V, M, _ = oi.shape
    for v in range(V):
        for i in np.flatnonzero(oi[v, :, 0]):
            x0, x1, y0, y1 = oi[v, i, 5:9]
            for ty in range(y0, y1 + 1):
                for tx in range(x0, x1 + 1):
                    lists.setdefault((v * ty_n + ty) * tx_n + tx, []).append(int(i))
    return {k: np.array(sorted(vv), dtype=np.int64) for k, vv in lists.items()}


def brick_bounds_f32(G, gdescs, Q3=11.345, B=8):
    """FP32 replica of the brick bound: [G, M, 13] = valid, voxel lo(3), hi(3), brick lo(3), hi(3)."""
    M = int(np.asarray(G.mean).shape[0])
    mean, scale, quat = _f(G.mean), _f(G.scale), _f(G.quat)
    gd = _f(np.atleast_2d(gdescs))
    out = np.zeros((gd.shape[0], M, 13), dtype=np.int32)
    lib().orc_brick_bounds_f32(M, _p(mean, _F), _p(scale, _F), _p(quat, _F), _p(gd, _F), gd.shape[0],
                               float(Q3), int(B), _p(out, _I))
    return out


def brick_lists_f32(G, gdescs, Q3=11.345, B=8):
    """Per-brick Gaussian lists: dict brick_key -> sorted ids, brick_key counted over
    grids in order, bricks of one grid in (bz, by, bx) row-major order."""
    bb = brick_bounds_f32(G, gdescs, Q3, B)
    gd = np.atleast_2d(gdescs)
    lists: dict[int, list[int]] = {}
    base = 0
    for g in range(gd.shape[0]):
        nb = [(int(gd[g][6 + k]) + B - 1) // B for k in range(3)]
        for i in np.flatnonzero(bb[g, :, 0]):
            bl, bh = bb[g, i, 7:10], bb[g, i, 10:13]
            for bz in range(bl[2], bh[2] + 1):
                for by in range(bl[1], bh[1] + 1):
                    for bx in range(bl[0], bh[0] + 1):
                        lists.setdefault(base + (bz * nb[1] + by) * nb[0] + bx, []).append(int(i))
        base += nb[0] * nb[1] * nb[2]
    return {k: np.array(sorted(v), dtype=np.int64) for k, v in lists.items()}
