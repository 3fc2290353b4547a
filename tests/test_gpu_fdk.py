"""Parity of the FDK initialisation kernels (Sec. 4.1) with the FP64 oracle: row
filtering, back-projection, the seeded draw of positions and the 3-NN scales."""
import math

import numpy as np
import pytest
import torch

from gpu_util import dev, host
from oracle import fdk
from paper_2405_20693_b300 import build, engine, r2g
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    r2g.lib()


def _filter_gpu(proj, cam):
    p = dev(proj)
    out = torch.empty_like(p)
    r2g.r2g_fdk_filter(p, r2g.camera(cam), out)
    return host(out)


def _f32grid(gd):
    return np.asarray(gd, np.float32).astype(np.float64)


@pytest.mark.parametrize("beam,W", [(1, 37), (1, 512), (0, 64), (1, 1), (1, 9)])
def test_fdk_filter_matches_oracle(beam, W):
    """Ragged rows (not a multiple of the 8 outputs per thread), a full 512-pixel
    row, a one-pixel row; cone pre-weighting with a detector offset."""
    H = 5
    cam = I.cone_camera(H, W, pitch=I.CONE_PITCH * 4) if beam else I.parallel_camera(H, W, 2.0 / W)
    cam.off_u = 0.3 * cam.pitch_u
    cam.off_v = -0.7 * cam.pitch_v
    proj = I.rng(W).uniform(0, 2, (3, H, W)).astype(np.float32)
    got = _filter_gpu(proj, cam)
    ref = fdk.fdk_filter(proj, cam)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("case", ["cone", "parallel", "cone_near", "cone_tilted"])
def test_fdk_backproject_matches_oracle(case):
    """A ragged 19 x 23 x 13 grid (not a multiple of the 32 x 8 x 8 thread tile), 7
    views of a phantom's filtered projections.  cone_near puts the near plane at the
    source-to-isocentre distance so each view skips the voxels on the source's side;
    cone_tilted tilts the orbit so u0 and u2 vary along z (the general path)."""
    ph, _ = I.normalised_phantom(3, 32)
    cam = I.cone_camera(40, 48, pitch=I.CONE_PITCH * 512 / 48) if case != "parallel" else \
        I.parallel_camera(40, 48, 2.4 / 48)
    views = I.view_table(np.deg2rad(np.arange(7) * 51.0 + 5.0), I.CONE_L_SO)
    if case == "cone_near":
        cam.near_plane = I.CONE_L_SO
    if case == "cone_tilted":
        c, s = math.cos(0.3), math.sin(0.3)
        tilt = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
        for v in range(7):
            views[v, :9] = (views[v, :9].reshape(3, 3).astype(np.float64) @ tilt).ravel().astype(np.float32)
    proj = I.phantom_projections(ph, views, cam).astype(np.float32)
    F = fdk.fdk_filter(proj, cam)
    Fd = dev(F)
    gd = _f32grid(I.grid_desc((-0.9, -0.8, -0.7), (0.09, 0.07, 0.11), (19, 23, 13)))
    vol = torch.empty((13, 23, 19), dtype=torch.float32, device="cuda")
    r2g.r2g_fdk_backproject(dev(views), r2g.camera(cam), Fd, r2g.grids(gd)[0], 2 * np.pi / 7, vol)
    ref = fdk.fdk_backproject(F.astype(np.float32), views, cam, gd, 2 * np.pi / 7)
    got = host(vol).ravel()
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    if case == "cone_near":
        assert (ref == 0).sum() == 0 or np.array_equal(got[ref == 0], ref[ref == 0])


def test_fdk_reconstructs_cylinder_on_gpu():
    """The z-invariant cylinder of the oracle pin, on the CUDA path: 1 inside, 0 outside."""
    cyl = I.Phantom(np.zeros((1, 3)), np.array([[0.5, 0.5, 30.0]]), np.eye(3)[None], np.array([1.0]))
    cam = I.cone_camera(96, 128, pitch=I.CONE_PITCH * 4)
    views = I.view_table(I.even_angles(180), I.CONE_L_SO)
    proj = I.phantom_projections(cyl, views, cam, device="cuda").astype(np.float32)
    vol = host(engine.fdk_volume(dev(views), dev(proj), cam, I.cube_grid(40)))
    xs = -1 + (np.arange(40) + 0.5) * 2 / 40
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    r2 = X ** 2 + Y ** 2
    inside = (r2 < 0.4 ** 2) & (np.abs(Z) < 0.5)
    outside = (r2 > 0.6 ** 2) & (r2 < 0.9 ** 2) & (np.abs(Z) < 0.5)
    assert abs(vol[inside].mean() - 1) < 2e-3 and np.abs(vol[inside] - 1).max() < 5e-3
    assert np.abs(vol[outside]).max() < 0.03


def test_fdk_full_size_sampled():
    """The FDK of the one-scan workload (50 cone-beam views of 512^2 -> 256^3), sampled:
    400 voxels on two z planes, against the oracle's filter (only the rows those voxels
    read) and back-projection at those voxel centres."""
    ph, _ = I.normalised_phantom(0, 64)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(50), I.CONE_L_SO)
    proj = I.phantom_projections(ph, views, cam, device="cuda").astype(np.float32)
    gd = I.cube_grid(256)
    vol = host(engine.fdk_volume(dev(views), dev(proj), cam, gd))
    g = I.rng(9)
    zs = (96, 161)
    pick = [(z, int(y), int(x)) for z in zs for y, x in g.integers(0, 256, (200, 2))]
    centres = fdk.voxel_centres(_f32grid(gd)).reshape(256, 256, 256, 3)
    pts = np.array([centres[z, y, x] for z, y, x in pick])
    # the detector rows those points read in each view (plus one for the bilinear step)
    rows = np.zeros((50, 512), bool)
    for v in range(50):
        Wm, t = views[v, :9].astype(np.float64).reshape(3, 3), views[v, 9:].astype(np.float64)
        u = pts @ Wm.T + t
        yc = (cam.L_SD * u[:, 1] / u[:, 2] - cam.off_v) / cam.pitch_v + 256 - 0.5
        for y0 in np.floor(yc).astype(int):
            rows[v, max(0, y0 - 1):min(512, y0 + 3)] = True
    F = fdk.fdk_filter(proj, cam, rows=rows)
    ref = fdk.fdk_backproject(np.nan_to_num(F), views, cam, gd, 2 * np.pi / 50, points=pts)
    got = np.array([vol[z, y, x] for z, y, x in pick])
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(vol).max()


def _init_pair(vol, gd, tau, M, seed, k):
    gdf = _f32grid(gd)
    g = r2g.grids(gdf)[0]
    mean = torch.empty((M, 3), device="cuda")
    scale = torch.empty((M, 3), device="cuda")
    quat = torch.empty((M, 4), device="cuda")
    rho = torch.empty(M, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(r2g.r2g_init_workspace_size(g, M), dtype=torch.uint8, device="cuda")
    r2g.r2g_init_gaussians(dev(vol), g, tau, M, seed, k, mean, scale, quat, rho, n_out, ws)
    n = int(n_out.item())
    got = tuple(host(t[:n]) for t in (mean, scale, quat, rho))
    idx = fdk.sample_candidates(np.asarray(vol, np.float32), tau, M, seed)
    return got, idx, gdf


def _check_init(got, idx, gdf, vol, k):
    mean, scale, quat, rho = got
    assert mean.shape[0] == idx.size
    ref_mean = fdk.voxel_centres(gdf)[idx]
    assert np.abs(mean - ref_mean).max() <= 1e-6 * max(1.0, np.abs(ref_mean).max())
    assert np.array_equal(quat, np.tile([1.0, 0, 0, 0], (idx.size, 1)))
    vv = np.asarray(vol, np.float32).ravel()[idx].astype(np.float64)
    assert np.abs(rho - k * vv).max() <= 1e-6 * np.abs(k * vv).max()
    return ref_mean


@pytest.mark.parametrize("M,seed", [(3000, 11), (1, 4), (10 ** 6, 2)])
def test_init_gaussians_matches_oracle(M, seed):
    """A seeded phantom volume (64^3 with noise) as the input of both sides: the same
    voxels are drawn (the keys and the threshold decision are exact on both), in the
    same order, with the same densities, and the same 3-NN scales.  M = 10^6 exceeds
    the candidates (every candidate is taken); M = 1 leaves a lone position."""
    _, vol = I.normalised_phantom(5, 64)
    vol = (vol + I.rng(seed).normal(0, 0.02, vol.shape)).astype(np.float32)
    gd = I.cube_grid(64)
    got, idx, gdf = _init_pair(vol, gd, 0.05, M, seed, 0.15)
    ref_mean = _check_init(got, idx, gdf, vol, 0.15)
    if M > idx.size:
        assert np.array_equal(idx, np.flatnonzero(vol.ravel() > np.float32(0.05)))
    ref_scale = fdk.knn3_mean_distance(ref_mean, lone=float(np.min(gdf[3:6])))
    assert np.abs(got[1][:, 0] - ref_scale).max() <= 1e-5 * ref_scale.max()
    assert np.array_equal(got[1][:, 0], got[1][:, 1]) and np.array_equal(got[1][:, 0], got[1][:, 2])


def test_init_gaussians_tiny_grid():
    """Three candidates on a 4 x 3 x 2 grid with unequal voxel edges: each takes the
    mean distance to the two others."""
    vol = np.zeros((2, 3, 4), np.float32)
    vol[0, 0, 0], vol[1, 2, 3], vol[0, 1, 2] = 0.5, 0.7, 0.9
    gd = I.grid_desc((-0.2, -0.3, -0.1), (0.1, 0.2, 0.3), (4, 3, 2))
    got, idx, gdf = _init_pair(vol, gd, 0.05, 8, 1, 0.15)
    ref_mean = _check_init(got, idx, gdf, vol, 0.15)
    assert idx.size == 3
    ref_scale = fdk.knn3_mean_distance(ref_mean)
    assert np.abs(got[1][:, 0] - ref_scale).max() <= 1e-6 * ref_scale.max()


def test_init_gaussians_full_size():
    """The paper's setting (M = 50k, tau = 0.05, k = 0.15) on a 256^3 volume (the
    seeded phantom with noise, the same float32 input on both sides): the drawn
    voxels, their order and densities exactly as the oracle draws them; the scales
    of 500 drawn positions against the oracle's brute force."""
    _, vol = I.normalised_phantom(0, 256)
    vol = (vol + I.rng(8).normal(0, 0.02, vol.shape)).astype(np.float32)
    gd = I.cube_grid(256)
    got, idx, gdf = _init_pair(vol, gd, engine.INIT_TAU, engine.INIT_M, 3, engine.INIT_K)
    assert idx.size == engine.INIT_M
    ref_mean = _check_init(got, idx, gdf, vol, engine.INIT_K)
    q = I.rng(3).choice(idx.size, 500, replace=False)
    ref_scale = fdk.knn3_mean_distance(ref_mean, which=q)
    assert np.abs(got[1][q, 0] - ref_scale).max() <= 1e-5 * ref_scale.max()


def test_fdk_init_composes_volume_and_draw():
    """fdk_init on the one-scan workload (50 views of 512^2 -> 256^3, M = 50k):
    M Gaussians at distinct voxel centres whose FDK value exceeds tau, in increasing
    voxel order, rho = k times that value, positive isotropic scales."""
    ph, _ = I.normalised_phantom(0, 64)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(50), I.CONE_L_SO)
    proj = I.phantom_projections(ph, views, cam, device="cuda").astype(np.float32)
    G, vol_dev = engine.fdk_init(dev(views), dev(proj), cam, 256, seed=3)
    vol = host(vol_dev).ravel()
    assert G.M == engine.INIT_M
    ijk = np.rint((G.mean + 1) * 128 - 0.5).astype(np.int64)
    assert np.abs(ijk - ((G.mean + 1) * 128 - 0.5)).max() < 1e-3
    j = (ijk[:, 2] * 256 + ijk[:, 1]) * 256 + ijk[:, 0]
    assert np.all(np.diff(j) > 0)
    assert np.all(vol[j] > np.float32(engine.INIT_TAU))
    assert np.abs(G.rho - engine.INIT_K * vol[j]).max() <= 1e-6
    assert np.all(G.scale > 0) and np.array_equal(G.scale[:, 0], G.scale[:, 2])
