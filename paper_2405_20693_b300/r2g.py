"""Thin ctypes binding of libr2g.so (the C ABI in include/r2g.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, takes torch CUDA tensors (or plain numbers / the ctypes structs
below), passes raw device pointers and the current torch stream, and raises
``R2GError`` on a non-OK status.  All computation happens in the CUDA library;
there is no fallback -- if libr2g.so is missing, importing this module works but
the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libr2g.so")

R2G_OK, R2G_E_INVAL, R2G_E_CAPACITY, R2G_E_CUDA, R2G_E_TIMEOUT, R2G_E_NUMERIC = range(6)
_NAMES = {0: "OK", 1: "E_INVAL", 2: "E_CAPACITY", 3: "E_CUDA", 4: "E_TIMEOUT", 5: "E_NUMERIC"}


class R2GError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"r2g {_NAMES.get(status, status)}: {msg}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("L_SD", ctypes.c_float),
                ("pitch_u", ctypes.c_float), ("pitch_v", ctypes.c_float), ("off_u", ctypes.c_float),
                ("off_v", ctypes.c_float), ("near_plane", ctypes.c_float)]


class RasterOpts(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_float), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("count_pairs", ctypes.c_int32), ("biased", ctypes.c_int32), ("separate_lists", ctypes.c_int32),
                ("dilation", ctypes.c_float), ("view_chunk", ctypes.c_int32)]


class DensifyOpts(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("min_density", ctypes.c_float), ("split_scale", ctypes.c_float),
                ("split_factor", ctypes.c_float), ("seed", ctypes.c_uint64)]


def densify_opts(grad_threshold=5e-5, min_density=1e-5, split_scale=0.02, split_factor=1.6, seed=0) -> DensifyOpts:
    return DensifyOpts(float(grad_threshold), float(min_density), float(split_scale), float(split_factor),
                       int(seed) & (2 ** 64 - 1))


class Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float * 3), ("dims", ctypes.c_int32 * 3)]


class AdamOpts(ctypes.Structure):
    _fields_ = [("lr0", ctypes.c_float * 4), ("final_factor", ctypes.c_float), ("total_iters", ctypes.c_int32),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class RoundEntry(ctypes.Structure):
    _fields_ = [("view", ctypes.c_int32), ("it", ctypes.c_int32), ("origin", ctypes.c_float * 3),
                ("pad", ctypes.c_int32 * 3)]


class Job(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("raw", ctypes.c_void_p), ("act", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("V", ctypes.c_int32), ("views", ctypes.c_void_p), ("meas", ctypes.c_void_p), ("cam", Camera),
                ("ropts", RasterOpts), ("Q3", ctypes.c_float), ("D", ctypes.c_int32), ("voxel", ctypes.c_float),
                ("lambda_ssim", ctypes.c_float), ("lambda_tv", ctypes.c_float), ("adam", AdamOpts),
                ("image", ctypes.c_void_p), ("dimage", ctypes.c_void_p), ("vol", ctypes.c_void_p),
                ("dvol", ctypes.c_void_p), ("loss", ctypes.c_void_p), ("raster_ws", ctypes.c_void_p),
                ("raster_ws_bytes", ctypes.c_size_t), ("voxel_ws", ctypes.c_void_p),
                ("voxel_ws_bytes", ctypes.c_size_t), ("loss_ws", ctypes.c_void_p),
                ("loss_ws_bytes", ctypes.c_size_t), ("tv_ws", ctypes.c_void_p), ("tv_ws_bytes", ctypes.c_size_t),
                ("dens_grad", ctypes.c_void_p), ("dens_count", ctypes.c_void_p), ("tv_eps", ctypes.c_float),
                ("views_per_step", ctypes.c_int32), ("n_patches", ctypes.c_int32), ("patch_origins", ctypes.c_void_p),
                ("full_vol", ctypes.c_void_p), ("full_grid", Grid), ("full_ws", ctypes.c_void_p),
                ("full_ws_bytes", ctypes.c_size_t)]


class Staging(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("meas", ctypes.c_void_p), ("views", ctypes.c_void_p),
                ("entries", ctypes.c_void_p), ("entries_host", ctypes.c_void_p), ("loss", ctypes.c_void_p),
                ("patch_origins", ctypes.c_void_p)]


def camera(cam) -> Camera:
    """Camera struct from an ``inputs.Camera``-like object."""
    return Camera(int(cam.beam), int(cam.H), int(cam.W), float(cam.L_SD), float(cam.pitch_u), float(cam.pitch_v),
                  float(cam.off_u), float(cam.off_v), float(cam.near_plane))


def raster_opts(Q=9.0, tile=(16, 16), count_pairs=False, biased=False, separate_lists=False,
                dilation=0.0, view_chunk=0) -> RasterOpts:
    return RasterOpts(float(Q), int(tile[0]), int(tile[1]), int(bool(count_pairs)), int(bool(biased)),
                      int(bool(separate_lists)), float(dilation), int(view_chunk))


def grids(gdescs) -> ctypes.Array:
    """Array of Grid structs from [G, 9] descriptors (origin, voxel, dims)."""
    import numpy as np

    gd = np.atleast_2d(np.asarray(gdescs, dtype=np.float64))
    arr = (Grid * gd.shape[0])()
    for g in range(gd.shape[0]):
        for k in range(3):
            arr[g].origin[k] = float(gd[g, k])
            arr[g].voxel[k] = float(gd[g, 3 + k])
            arr[g].dims[k] = int(gd[g, 6 + k])
    return arr


def adam_opts(lr0=(2e-4, 5e-3, 1e-3, 1e-2), final_factor=0.1, total_iters=30000, beta1=0.9, beta2=0.999,
              eps=1e-15) -> AdamOpts:
    return AdamOpts((ctypes.c_float * 4)(*lr0), final_factor, total_iters, beta1, beta2, eps)


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_F = ctypes.c_float
_SZ = ctypes.c_size_t


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built (run paper_2405_20693_b300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "r2g_raster_workspace_size": (_SZ, [_I64, _I32, _P, _P, _I64]),
            "r2g_rasterize": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _SZ, _P]),
            "r2g_rasterize_backward": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ,
                                              _P]),
            "r2g_project": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P]),
            "r2g_mean_mu": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P]),
            "r2g_fdk_filter": (_I32, [_I32, _P, _P, _P, _P]),
            "r2g_fdk_backproject": (_I32, [_I32, _P, _P, _P, _P, ctypes.c_float, _P, _P]),
            "r2g_init_workspace_size": (_SZ, [_P, _I64]),
            "r2g_metrics_workspace_size": (_SZ, [_I32, _I32, _I32]),
            "r2g_densify_workspace_size": (_SZ, []),
            "r2g_densify": (_I32, [_I64, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P]),
            "r2g_volume_metrics": (_I32, [_I32, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
            "r2g_init_gaussians": (_I32, [_P, _P, ctypes.c_float, _I64, ctypes.c_uint64, ctypes.c_float, _P, _P, _P,
                                          _P, _P, _P, _SZ, _P]),
            "r2g_raster_lists": (_I32, [_I64, _I32, _P, _P, _P, _SZ, _P, _P, _I64, _P, _P]),
            "r2g_pair_count": (_I32, [_P, _SZ, _P, _P]),
            "r2g_voxel_workspace_size": (_SZ, [_I64, _I32, _P, _I64]),
            "r2g_voxelize": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _F, _P, _P, _SZ, _P]),
            "r2g_voxelize_counted": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _F, _P, _P, _SZ, _P]),
            "r2g_voxelize_backward": (_I32, [_I64, _P, _P, _P, _P, _I32, _P, _F, _P, _P, _P, _P, _P, _P, _SZ, _P]),
            "r2g_voxel_lists": (_I32, [_I64, _I32, _P, _P, _SZ, _P, _P, _I64, _P, _P]),
            "r2g_loss_workspace_size": (_SZ, [_I32, _I32, _I32]),
            "r2g_projection_loss": (_I32, [_I32, _I32, _I32, _P, _P, _F, _P, _P, _P, _SZ, _P]),
            "r2g_tv_workspace_size": (_SZ, [_I32, _I32]),
            "r2g_tv3d": (_I32, [_I32, _I32, _P, _F, _P, _P, _P, _SZ, _P]),
            "r2g_tv3d_noalloc": (_I32, [_I32, _I32, _P, _F, _P, _P, _P]),
            "r2g_tv3d_iso": (_I32, [_I32, _I32, _P, _F, _F, _P, _P, _P, _SZ, _P]),
            "r2g_adam_step": (_I32, [_I64, _P, _P, _P, _P, _P, _I32, _P, _P]),
            "r2g_poll": (_I32, [_P, _SZ, _P, _P]),
            "r2g_set_wait_limit": (_I32, [ctypes.c_uint64]),
            "r2g_train_step": (_I32, [_P, _P, _P]),
            "r2g_train_step_host": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _P]),
            "r2g_train_step_host_batch": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _P, _P]),
            "r2g_train_step_host_wait": (_I32, [_P, _I64, _P]),
            "r2g_upload_round": (_I32, [_P, _P, _I32, _P]),
            "r2g_profile_enable": (_I32, [_I32, _I32]),
            "r2g_profile_select": (_I32, [ctypes.c_uint32]),
            "r2g_profile_reset": (_I32, []),
            "r2g_profile_read": (_I32, [_I32, _P, _P]),
            "r2g_profile_name": (ctypes.c_char_p, [_I32]),
            "r2g_launch_count": (_I64, []),
            "r2g_last_error": (ctypes.c_char_p, []),
            "r2g_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("r2g_")]


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("tensors passed to libr2g must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensors passed to libr2g must be contiguous")
    return t.data_ptr()


def _f32(*ts):
    for t in ts:
        if t is not None and t.dtype != torch.float32:
            raise ValueError("float32 tensors required")


def _gp(grid_arr):
    return ctypes.cast(grid_arr, ctypes.c_void_p)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(status: int):
    if status != R2G_OK:
        raise R2GError(status, lib().r2g_last_error().decode())


def last_error() -> str:
    """The library's message for the last failure on this thread."""
    return lib().r2g_last_error().decode()


# ----------------------------------------------------------------------------- rasterizer


def r2g_raster_workspace_size(M: int, V: int, cam: Camera, opts: RasterOpts, key_capacity: int) -> int:
    n = lib().r2g_raster_workspace_size(M, V, ctypes.byref(cam), ctypes.byref(opts), key_capacity)
    if n == 0:
        raise R2GError(R2G_E_INVAL, lib().r2g_last_error().decode())
    return int(n)


def r2g_rasterize(mean, scale, quat, rho, views, cam: Camera, opts: RasterOpts, image, ws, stream=None):
    _f32(mean, scale, quat, rho, views, image)
    M, V = mean.shape[0], views.shape[0]
    _check(lib().r2g_rasterize(M, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho), V, _ptr(views),
                               ctypes.byref(cam), ctypes.byref(opts), _ptr(image), _ptr(ws), ws.numel(),
                               _stream(stream)))


def r2g_rasterize_backward(mean, scale, quat, rho, views, cam: Camera, opts: RasterOpts, dimage, dmean, dscale,
                           dquat, drho, ws, stream=None):
    _f32(mean, scale, quat, rho, views, dimage, dmean, dscale, dquat, drho)
    M, V = mean.shape[0], views.shape[0]
    _check(lib().r2g_rasterize_backward(M, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho), V, _ptr(views),
                                        ctypes.byref(cam), ctypes.byref(opts), _ptr(dimage), _ptr(dmean),
                                        _ptr(dscale), _ptr(dquat), _ptr(drho), _ptr(ws), ws.numel(),
                                        _stream(stream)))


def r2g_project(mean, scale, quat, rho, views, cam: Camera, opts: RasterOpts, proj, rect, stream=None):
    _f32(mean, scale, quat, rho, views, proj)
    M, V = mean.shape[0], views.shape[0]
    _check(lib().r2g_project(M, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho), V, _ptr(views), ctypes.byref(cam),
                             ctypes.byref(opts), _ptr(proj), _ptr(rect), _stream(stream)))


def r2g_mean_mu(mean, scale, quat, views, cam: Camera, mu_mean=None, rho=None, rho_vol=None, stream=None):
    _f32(mean, scale, quat, views, mu_mean, rho, rho_vol)
    M, V = mean.shape[0], views.shape[0]
    _check(lib().r2g_mean_mu(M, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho), V, _ptr(views), ctypes.byref(cam),
                             _ptr(mu_mean), _ptr(rho_vol), _stream(stream)))


def r2g_fdk_filter(proj, cam: Camera, filt, stream=None):
    _f32(proj, filt)
    _check(lib().r2g_fdk_filter(proj.shape[0], ctypes.byref(cam), _ptr(proj), _ptr(filt), _stream(stream)))


def r2g_fdk_backproject(views, cam: Camera, filt, grid, dbeta: float, vol, stream=None):
    """grid: one Grid struct (see grids())."""
    _f32(views, filt, vol)
    _check(lib().r2g_fdk_backproject(views.shape[0], _ptr(views), ctypes.byref(cam), _ptr(filt), ctypes.byref(grid),
                                     float(dbeta), _ptr(vol), _stream(stream)))


def r2g_init_workspace_size(grid, M: int) -> int:
    return lib().r2g_init_workspace_size(ctypes.byref(grid), int(M))


def r2g_init_gaussians(vol, grid, tau: float, M: int, seed: int, k: float, mean, scale, quat, rho, n_out, ws,
                       stream=None):
    _f32(vol, mean, scale, quat, rho)
    if n_out.dtype != torch.int64:
        raise ValueError("n_out must be an int64 tensor")
    _check(lib().r2g_init_gaussians(_ptr(vol), ctypes.byref(grid), float(tau), int(M), int(seed) & (2 ** 64 - 1),
                                    float(k), _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho), _ptr(n_out), _ptr(ws),
                                    ws.numel(), _stream(stream)))


def r2g_densify_workspace_size() -> int:
    return lib().r2g_densify_workspace_size()


def r2g_densify(M: int, raw, act, m, v, dens_grad, dens_count, opts: DensifyOpts, max_gaussians: int, raw_out,
                act_out, m_out, v_out, m_new, ws, stream=None):
    _f32(raw, act, m, v, dens_grad, dens_count, raw_out, act_out, m_out, v_out)
    if m_new.dtype != torch.int64:
        raise ValueError("m_new must be an int64 tensor")
    _check(lib().r2g_densify(int(M), _ptr(raw), _ptr(act), _ptr(m), _ptr(v), _ptr(dens_grad), _ptr(dens_count),
                             ctypes.byref(opts), int(max_gaussians), _ptr(raw_out), _ptr(act_out), _ptr(m_out),
                             _ptr(v_out), _ptr(m_new), _ptr(ws), ws.numel(), _stream(stream)))


def r2g_metrics_workspace_size(X: int, Y: int, Z: int) -> int:
    return lib().r2g_metrics_workspace_size(int(X), int(Y), int(Z))


def r2g_volume_metrics(vol, ref, out, ws, stream=None):
    """vol, ref: float32 [Z, Y, X]; out: float64 [6] = MSE, PSNR, SSIM, axial, coronal, sagittal."""
    _f32(vol, ref)
    if out.dtype != torch.float64:
        raise ValueError("out must be a float64 tensor")
    Z, Y, X = vol.shape
    _check(lib().r2g_volume_metrics(X, Y, Z, _ptr(vol), _ptr(ref), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))


def r2g_raster_lists(M: int, V: int, cam: Camera, opts: RasterOpts, ws, ranges, ids, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check(lib().r2g_raster_lists(M, V, ctypes.byref(cam), ctypes.byref(opts), _ptr(ws), ws.numel(), _ptr(ranges),
                                  _ptr(ids), ids.numel(), ctypes.byref(n), _stream(stream)))
    return int(n.value)


def r2g_pair_count(ws, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check(lib().r2g_pair_count(_ptr(ws), ws.numel(), ctypes.byref(n), _stream(stream)))
    return int(n.value)


def r2g_poll(ws, stream=None) -> tuple[int, int]:
    """(status, needed entries); the device statuses (R2G_E_CAPACITY, R2G_E_TIMEOUT,
    R2G_E_NUMERIC) are returned, not raised."""
    n = ctypes.c_int64(0)
    st = lib().r2g_poll(_ptr(ws), ws.numel(), _stream(stream), ctypes.byref(n))
    if st not in (R2G_OK, R2G_E_CAPACITY, R2G_E_TIMEOUT, R2G_E_NUMERIC):
        _check(st)
    return int(st), int(n.value)


def r2g_set_wait_limit(polls: int):
    """Polls before a device-side wait gives up (0: the default)."""
    _check(lib().r2g_set_wait_limit(ctypes.c_uint64(int(polls))))


# ----------------------------------------------------------------------------- voxelizer


def r2g_voxel_workspace_size(M: int, grid_arr, key_capacity: int) -> int:
    n = lib().r2g_voxel_workspace_size(M, len(grid_arr), _gp(grid_arr), key_capacity)
    if n == 0:
        raise R2GError(R2G_E_INVAL, "bad voxel workspace arguments")
    return int(n)


def r2g_voxelize(mean, scale, quat, rho, grid_arr, Q3, vol, ws, stream=None, counted=False):
    _f32(mean, scale, quat, rho, vol)
    f = lib().r2g_voxelize_counted if counted else lib().r2g_voxelize
    _check(f(mean.shape[0], _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho), len(grid_arr), _gp(grid_arr), float(Q3),
             _ptr(vol), _ptr(ws), ws.numel(), _stream(stream)))


def r2g_voxelize_backward(mean, scale, quat, rho, grid_arr, Q3, dvol, dmean, dscale, dquat, drho, ws,
                          stream=None):
    _f32(mean, scale, quat, rho, dvol, dmean, dscale, dquat, drho)
    _check(lib().r2g_voxelize_backward(mean.shape[0], _ptr(mean), _ptr(scale), _ptr(quat), _ptr(rho),
                                       len(grid_arr), _gp(grid_arr), float(Q3), _ptr(dvol), _ptr(dmean), _ptr(dscale),
                                       _ptr(dquat), _ptr(drho), _ptr(ws), ws.numel(), _stream(stream)))


def r2g_voxel_lists(M: int, grid_arr, ws, ranges, ids, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check(lib().r2g_voxel_lists(M, len(grid_arr), _gp(grid_arr), _ptr(ws), ws.numel(), _ptr(ranges), _ptr(ids),
                                 ids.numel(), ctypes.byref(n), _stream(stream)))
    return int(n.value)


# ----------------------------------------------------------------------------- losses, optimizer


def r2g_loss_workspace_size(V: int, H: int, W: int) -> int:
    return int(lib().r2g_loss_workspace_size(V, H, W))


def r2g_projection_loss(render, meas, lambda_ssim, loss, drender, ws, stream=None):
    _f32(render, meas, loss, drender)
    V, H, W = render.shape
    _check(lib().r2g_projection_loss(V, H, W, _ptr(render), _ptr(meas), float(lambda_ssim), _ptr(loss),
                                     _ptr(drender), _ptr(ws), ws.numel(), _stream(stream)))


def r2g_tv_workspace_size(G: int, D: int) -> int:
    return int(lib().r2g_tv_workspace_size(G, D))


def r2g_tv3d(vol, lambda_tv, loss, dvol, ws, stream=None):
    _f32(vol, loss, dvol)
    G, D = vol.shape[0], vol.shape[1]
    _check(lib().r2g_tv3d(G, D, _ptr(vol), float(lambda_tv), _ptr(loss), _ptr(dvol), _ptr(ws), ws.numel(),
                          _stream(stream)))


def r2g_tv3d_iso(vol, lambda_tv, eps, loss, dvol, ws, stream=None):
    _f32(vol, loss, dvol)
    G, D = vol.shape[0], vol.shape[1]
    _check(lib().r2g_tv3d_iso(G, D, _ptr(vol), float(lambda_tv), float(eps), _ptr(loss), _ptr(dvol), _ptr(ws),
                              ws.numel(), _stream(stream)))


def r2g_tv3d_noalloc(vol, lambda_tv, loss, dvol, stream=None):
    _f32(vol, loss, dvol)
    G, D = vol.shape[0], vol.shape[1]
    _check(lib().r2g_tv3d_noalloc(G, D, _ptr(vol), float(lambda_tv), _ptr(loss), _ptr(dvol), _stream(stream)))


def r2g_adam_step(raw, act, grad, m, v, it: int, opts: AdamOpts, stream=None):
    _f32(raw, act, grad, m, v)
    M = raw.numel() // 11
    _check(lib().r2g_adam_step(M, _ptr(raw), _ptr(act), _ptr(grad), _ptr(m), _ptr(v), int(it), ctypes.byref(opts),
                               _stream(stream)))


PROFILE_KERNELS = ("project", "emit", "sort", "ranges", "splat_fwd", "splat_bwd", "project_bwd", "vox_project",
                   "vox_fwd", "vox_bwd", "vox_chain", "loss", "tv", "adam", "vox_emit", "vox_sort", "vox_ranges",
                   "fdk_filter", "fdk_bp", "init_select", "init_knn", "metrics", "densify")


def r2g_profile_enable(on: bool, max_spans: int = 4096):
    _check(lib().r2g_profile_enable(int(on), int(max_spans)))


def r2g_profile_select(kernel_mask: int):
    _check(lib().r2g_profile_select(int(kernel_mask) & 0xFFFFFFFF))


def r2g_profile_reset():
    _check(lib().r2g_profile_reset())


def r2g_profile_read(kernel: int) -> tuple[int, float]:
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(lib().r2g_profile_read(int(kernel), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def r2g_profile_name(kernel: int) -> str:
    return lib().r2g_profile_name(int(kernel)).decode()


def r2g_launch_count() -> int:
    return int(lib().r2g_launch_count())


def r2g_train_step(job: Job, entry_ptr: int, stream=None):
    """One training iteration of one scan; entry_ptr is the device address of its
    round entry (r2g_round_entry)."""
    _check(lib().r2g_train_step(ctypes.byref(job), ctypes.c_void_p(int(entry_ptr)), _stream(stream)))


def r2g_train_step_host(job: Job, stg: Staging, step: int, meas_ptr: int, view_ptr: int, entry_ptr: int,
                        loss_ptr: int, stream=None):
    """One training iteration fed from host memory (addresses of the step's pinned
    measured projection, geometry row, round entry and 2-float loss buffer)."""
    _check(lib().r2g_train_step_host(ctypes.byref(job), ctypes.byref(stg), int(step), meas_ptr, view_ptr, entry_ptr,
                                     loss_ptr, _stream(stream)))


def r2g_train_step_host_batch(job: Job, stg: Staging, step: int, meas_ptr: int, views_ptr: int, origins_ptr,
                              entry_ptr: int, loss_ptr: int, stream=None):
    """The batch form of r2g_train_step_host: host addresses of the step's pinned
    measured projections [Vs][H][W], geometry rows [Vs][12], TV patch origins
    [n_patches][3] (or None for one patch), round entry and 2-float loss buffer."""
    _check(lib().r2g_train_step_host_batch(ctypes.byref(job), ctypes.byref(stg), int(step), meas_ptr, views_ptr,
                                           origins_ptr, entry_ptr, loss_ptr, _stream(stream)))


def r2g_train_step_host_wait(stg: Staging, step: int, stream=None):
    _check(lib().r2g_train_step_host_wait(ctypes.byref(stg), int(step), _stream(stream)))


def r2g_upload_round(dst_dev, src_pinned, n: int, stream=None):
    """Asynchronous copy of n round entries from a pinned host tensor to the device."""
    if not src_pinned.is_pinned():
        raise ValueError("the round table must be in page-locked host memory")
    _check(lib().r2g_upload_round(_ptr(dst_dev), ctypes.c_void_p(src_pinned.data_ptr()), int(n), _stream(stream)))


def r2g_version() -> str:
    return lib().r2g_version().decode()
