"""Host-side checks of the C ABI library that need no GPU: it builds for sm_103a,
loads, exports every entry point include/r2g.h declares, and rejects bad
arguments on the host before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2405_20693_b300 import build, r2g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return r2g.lib()


def declared():
    txt = open(os.path.join(ROOT, "include", "r2g.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(r2g_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = declared()
    for n in ("r2g_rasterize", "r2g_rasterize_backward", "r2g_voxelize", "r2g_voxelize_backward", "r2g_project"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", r2g.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (r2g_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    # nothing but the ABI is exported
    assert all(n in declared() for n in exported), sorted(exported - set(declared()))


def test_version_string(lib):
    assert "sm_103a" in r2g.r2g_version()


def test_host_side_argument_errors(lib):
    cam = r2g.Camera(1, 512, 512, 11.7, 0.00625, 0.00625, 0.0, 0.0, 0.078)
    bad_tile = r2g.raster_opts(9.0, (12, 12))
    assert lib.r2g_raster_workspace_size(1000, 1, ctypes.byref(cam), ctypes.byref(bad_tile), 4096) == 0
    assert "tile" in lib.r2g_last_error().decode()
    ok = r2g.raster_opts(9.0, (16, 16))
    n = lib.r2g_raster_workspace_size(1000, 1, ctypes.byref(cam), ctypes.byref(ok), 4096)
    assert n > 2 * 8 * 4096
    for bad in (-0.1, float("nan"), float("inf")):  # dilation must be finite and >= 0
        o = r2g.raster_opts(9.0, (16, 16), dilation=bad)
        assert lib.r2g_raster_workspace_size(1000, 1, ctypes.byref(cam), ctypes.byref(o), 4096) == 0
        assert "dilation" in lib.r2g_last_error().decode()
    assert lib.r2g_raster_workspace_size(1000, 1, ctypes.byref(cam),
                                         ctypes.byref(r2g.raster_opts(9.0, (16, 16), dilation=0.3)), 4096) == n
    # NULL pointers are rejected on the host with R2G_E_INVAL, nothing launched
    st = lib.r2g_rasterize(1000, None, None, None, None, 1, None, ctypes.byref(cam), ctypes.byref(ok), None, None,
                           0, None)
    assert st == r2g.R2G_E_INVAL
    g = r2g.grids([[-1, -1, -1, 0.1, 0.1, 0.1, 0, 20, 20]])
    assert lib.r2g_voxel_workspace_size(1000, 1, ctypes.cast(g, ctypes.c_void_p), 4096) == 0
    assert lib.r2g_tv_workspace_size(1, 1) == 0
    st = lib.r2g_tv3d(1, 1, None, 0.05, None, None, None, 0, None)
    assert st == r2g.R2G_E_INVAL
    stg = r2g.Staging(0, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000)  # n_slots 0: rejected before any CUDA call
    job = r2g.Job()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the argument checks fail first
    assert lib.r2g_train_step_host(ctypes.byref(job), ctypes.byref(stg), 0, fake, fake, fake, fake,
                                   None) == r2g.R2G_E_INVAL
    assert lib.r2g_train_step_host_wait(ctypes.byref(stg), 0, None) == r2g.R2G_E_INVAL
    st = lib.r2g_tv3d_iso(1, 4, fake, 0.05, 0.0, fake, fake, fake, 4096, None)
    assert st == r2g.R2G_E_INVAL


def test_host_side_argument_errors_of_the_other_entry_points(lib):
    """FDK initialisation, volume metrics, adaptive control and the mean-mu query
    reject bad arguments on the host (R2G_E_INVAL, or a zero workspace size)."""
    cam = r2g.Camera(1, 64, 64, 11.7, 0.05, 0.05, 0.0, 0.0, 0.078)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its host checks
    assert lib.r2g_fdk_filter(0, ctypes.byref(cam), fake, fake, None) == r2g.R2G_E_INVAL
    assert lib.r2g_fdk_filter(1, ctypes.byref(cam), None, fake, None) == r2g.R2G_E_INVAL
    assert lib.r2g_fdk_filter(1, ctypes.byref(cam), fake, fake, None) == r2g.R2G_E_INVAL  # aliased
    wide = r2g.Camera(1, 4, 9000, 11.7, 0.05, 0.05, 0.0, 0.0, 0.078)
    assert lib.r2g_fdk_filter(1, ctypes.byref(wide), fake, ctypes.c_void_p(0x2000), None) == r2g.R2G_E_INVAL
    bad = r2g.grids([[-1, -1, -1, 0.1, 0.1, 0.1, 0, 20, 20]])[0]
    good = r2g.grids([[-1, -1, -1, 0.1, 0.1, 0.1, 20, 20, 20]])[0]
    assert lib.r2g_fdk_backproject(1, fake, ctypes.byref(cam), fake, ctypes.byref(bad), 0.1, fake, None) == \
        r2g.R2G_E_INVAL
    assert lib.r2g_init_workspace_size(ctypes.byref(bad), 10) == 0
    assert lib.r2g_init_workspace_size(ctypes.byref(good), 0) == 0
    ws_n = lib.r2g_init_workspace_size(ctypes.byref(good), 10)
    assert ws_n > 0
    assert lib.r2g_init_gaussians(fake, ctypes.byref(good), 0.05, 10, 1, 0.15, fake, fake, fake, fake, fake, fake,
                                  ws_n - 1, None) == r2g.R2G_E_INVAL
    assert lib.r2g_init_gaussians(fake, ctypes.byref(good), 0.05, 10, 1, 0.15, fake, fake, ctypes.c_void_p(0x1004),
                                  fake, fake, fake, ws_n, None) == r2g.R2G_E_INVAL  # quat not 16-byte aligned
    assert lib.r2g_metrics_workspace_size(0, 4, 4) == 0
    assert lib.r2g_volume_metrics(4, 4, 5000, fake, fake, fake, fake, 1 << 20, None) == r2g.R2G_E_INVAL
    opts = r2g.densify_opts()
    assert lib.r2g_densify(100, fake, fake, fake, fake, fake, fake, ctypes.byref(opts), 99, fake, fake, fake, fake,
                           fake, fake, 4096, None) == r2g.R2G_E_INVAL  # max_gaussians < M
    assert lib.r2g_densify(100, fake, fake, fake, fake, fake, None, ctypes.byref(opts), 200, fake, fake, fake, fake,
                           fake, fake, 4096, None) == r2g.R2G_E_INVAL
    assert lib.r2g_densify(100, fake, fake, fake, fake, fake, fake, ctypes.byref(opts), 200, fake, fake, fake, fake,
                           fake, fake, 0, None) == r2g.R2G_E_INVAL  # workspace too small
    assert lib.r2g_mean_mu(10, fake, fake, fake, None, 1, fake, ctypes.byref(cam), None, None, None) == \
        r2g.R2G_E_INVAL
