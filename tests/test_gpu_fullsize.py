"""Parity at the full sizes of the benchmark and scale configurations, in the
launch configuration bench.py uses (16x16 tiles, 8^3 bricks, default gates)."""
import numpy as np
import pytest
import torch

from gpu_util import assert_grads_close, assert_values_close, config2, config3, dev, dev_set, host
from oracle import core
from paper_2405_20693_b300 import build, engine
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def test_one_scan_view_and_patch_full_size():
    """The bench workload: one 512^2 cone-beam view of 50k Gaussians and one 32^3 TV
    patch, forward against the oracle's full image/volume, backward against the
    oracle's adjoint."""
    G, cam, views, _, _ = config2()
    v = views[17:18]
    rast = engine.Rasterizer(G.M, 1, cam)
    mean, scale, quat, rho = dev_set(G)
    img = rast.forward(mean, scale, quat, rho, dev(v), count=True)
    ref, pairs, band = core.render(G, v, cam, Q=engine.Q_PIXEL, want_band=True)
    assert_values_close(host(img), ref, band, "one-scan view")
    assert abs(rast.pair_count() - pairs) <= max(10, 1e-4 * pairs)
    dimg = (I.rng(12).standard_normal(ref.shape) / ref.size).astype(np.float32)
    g = [torch.zeros_like(t) for t in (mean, scale, quat, rho)]
    rast.backward(mean, scale, quat, rho, dev(v), dev(dimg), *g)
    gref, band = core.render_backward(G, v, cam, dimg, Q=engine.Q_PIXEL, want_band=True)
    zero_scale = np.abs(gref[1]).max() * float(np.max(G.scale))  # rotations of isotropic Gaussians: exactly 0
    for name, a, b, bd in zip(("mean", "scale", "quat", "rho"), g, gref, band):
        assert_grads_close(host(a), b, f"one-scan d{name}", band=bd, zero_scale=zero_scale)
    gd = np.asarray(I.patch_grid((101, 57, 140), 32, 256), np.float32).astype(np.float64)
    vox = engine.Voxelizer(G.M, gd)
    vol = vox.forward(mean, scale, quat, rho)
    vref, _, vband = core.voxelize(G, gd, engine.Q_VOXEL, want_band=True)
    assert_values_close(host(vol), vref, vband, "TV patch")
    dvol = I.rng(13).standard_normal(vox.n_vox).astype(np.float32)
    g = [torch.zeros_like(t) for t in (mean, scale, quat, rho)]
    vox.backward(mean, scale, quat, rho, dev(dvol), *g)
    vg, vb = core.voxelize_backward(G, gd, dvol, engine.Q_VOXEL, want_band=True)
    zero_scale = np.abs(vg[1]).max() * float(np.max(G.scale))
    for name, a, b, bd in zip(("mean", "scale", "quat", "rho"), g, vg, vb):
        assert_grads_close(host(a), b, f"TV patch d{name}", band=bd, zero_scale=zero_scale)


def test_scale_config_sampled():
    """500k Gaussians, all 75 views rasterized in one launch: views 0 and 40 are
    compared pixel by pixel with the oracle; the 256^3 volume is compared on two
    sampled 8x8x8 sub-blocks (the oracle evaluates every Gaussian there)."""
    G, cam, views, _, _ = config3()
    rast = engine.Rasterizer(G.M, views.shape[0], cam)
    mean, scale, quat, rho = dev_set(G)
    img = rast.forward(mean, scale, quat, rho, dev(views))
    for v in (0, 40):
        ref, _, band = core.render(G, views[v:v + 1], cam, Q=engine.Q_PIXEL, want_band=True)
        assert_values_close(host(img[v:v + 1]), ref, band, f"scale view {v}")
    # the adjoint of all 75 views against the oracle on a 2,000-Gaussian subset, in the
    # same 75-view, 512^2 launch shape
    sub = G.subset(np.arange(2000))
    r2 = engine.Rasterizer(sub.M, views.shape[0], cam)
    sm, ss, sq, sr = dev_set(sub)
    r2.forward(sm, ss, sq, sr, dev(views))
    dimg = (I.rng(14).standard_normal((views.shape[0], cam.H, cam.W)) * 1e-4).astype(np.float32)
    g = [torch.zeros_like(t) for t in (sm, ss, sq, sr)]
    r2.backward(sm, ss, sq, sr, dev(views), dev(dimg), *g)
    gref, band = core.render_backward(sub, views, cam, dimg, Q=engine.Q_PIXEL, want_band=True)
    for name, a, b, bd in zip(("mean", "scale", "quat", "rho"), g, gref, band):
        assert_grads_close(host(a), b, f"scale d{name}", band=bd)
    gd = np.asarray(I.cube_grid(256), np.float32).astype(np.float64)
    vox = engine.Voxelizer(G.M, gd)
    vol = host(vox.forward(mean, scale, quat, rho)).reshape(256, 256, 256)
    # one block inside the phantom, one across the edge of its support
    for (z, y, x) in ((120, 128, 96), (144, 56, 112)):
        sub = np.asarray(I.grid_desc((-1 + x * 2 / 256, -1 + y * 2 / 256, -1 + z * 2 / 256), (2 / 256,) * 3,
                                     (8, 8, 8)), np.float32).astype(np.float64)
        ref, _, band = core.voxelize(G, sub, engine.Q_VOXEL, want_band=True)
        assert_values_close(vol[z:z + 8, y:y + 8, x:x + 8].ravel(), ref, band, f"volume block {z},{y},{x}")
