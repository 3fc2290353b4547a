"""Failure detection without a GPU fault: the grid barriers of the cooperative list
builds wait with a bound; a test shrinks the bound to one poll so that a wait runs
out (the blocks of a cooperative launch never all arrive within 20 ns), and checks
that every kernel of the call ends, that the status reads R2G_E_TIMEOUT, that the
list consumers did no work, and that the next call with the default bound is
exact again."""
import numpy as np
import pytest
import torch

from gpu_util import dev, dev_set, host
from paper_2405_20693_b300 import build, engine, r2g
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.fixture
def short_waits():
    r2g.r2g_set_wait_limit(1)
    yield
    r2g.r2g_set_wait_limit(0)


def _scene():
    ph, vol = I.normalised_phantom(0, 256)
    G = I.init_from_volume(vol, I.cube_grid(256), 20_000, 9)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(50), I.CONE_L_SO)[7:8]
    return G, cam, views


def test_raster_list_build_timeout_is_reported_and_recovers(short_waits):
    G, cam, views = _scene()
    mean, scale, quat, rho = dev_set(G)
    rast = engine.Rasterizer(G.M, 1, cam, tile=(16, 16))  # 1024 tiles: the cooperative build
    r2g.r2g_set_wait_limit(0)
    ref = host(rast.forward(mean, scale, quat, rho, dev(views)))
    r2g.r2g_set_wait_limit(1)
    img = torch.empty((1, cam.H, cam.W), dtype=torch.float32, device="cuda")
    rast.forward(mean, scale, quat, rho, dev(views), img, check=False)
    g = [torch.zeros_like(t) for t in (mean, scale, quat, rho)]
    rast.backward(mean, scale, quat, rho, dev(views), torch.ones_like(img), *g)
    torch.cuda.synchronize()  # every kernel of both calls ended
    assert r2g.r2g_poll(rast.ws)[0] == r2g.R2G_E_TIMEOUT
    # the backward's splat kernel skipped: no moment, so no gradient at all
    assert all(float(t.abs().max()) == 0.0 for t in g)
    r2g.r2g_set_wait_limit(0)
    again = host(rast.forward(mean, scale, quat, rho, dev(views)))
    assert r2g.r2g_poll(rast.ws)[0] == r2g.R2G_OK
    assert np.array_equal(again, ref)  # the forward is deterministic


def test_brick_list_build_timeout_is_reported_and_recovers(short_waits):
    G, _, _ = _scene()
    mean, scale, quat, rho = dev_set(G)
    gd = I.patch_grid((100, 90, 110), 32, 256)  # 64 bricks: the cooperative build
    vox = engine.Voxelizer(G.M, gd)
    r2g.r2g_set_wait_limit(0)
    ref = host(vox.forward(mean, scale, quat, rho))
    r2g.r2g_set_wait_limit(1)
    vol = torch.empty(32 ** 3, dtype=torch.float32, device="cuda")
    vox.forward(mean, scale, quat, rho, vol, check=False)
    g = [torch.zeros_like(t) for t in (mean, scale, quat, rho)]
    vox.backward(mean, scale, quat, rho, torch.ones_like(vol), *g)
    torch.cuda.synchronize()
    assert r2g.r2g_poll(vox.ws)[0] == r2g.R2G_E_TIMEOUT
    assert all(float(t.abs().max()) == 0.0 for t in g)
    r2g.r2g_set_wait_limit(0)
    again = host(vox.forward(mean, scale, quat, rho))
    assert r2g.r2g_poll(vox.ws)[0] == r2g.R2G_OK
    assert np.array_equal(again, ref)
