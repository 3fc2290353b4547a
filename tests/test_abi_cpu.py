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
    # NULL pointers are rejected on the host with R2G_E_INVAL, nothing launched
    st = lib.r2g_rasterize(1000, None, None, None, None, 1, None, ctypes.byref(cam), ctypes.byref(ok), None, None,
                           0, None)
    assert st == r2g.R2G_E_INVAL
    g = r2g.grids([[-1, -1, -1, 0.1, 0.1, 0.1, 0, 20, 20]])
    assert lib.r2g_voxel_workspace_size(1000, 1, ctypes.cast(g, ctypes.c_void_p), 4096) == 0
    assert lib.r2g_tv_workspace_size(1, 1) == 0
    st = lib.r2g_tv3d(1, 1, None, 0.05, None, None, None, 0, None)
    assert st == r2g.R2G_E_INVAL
