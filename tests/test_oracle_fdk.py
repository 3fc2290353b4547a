"""Pins of the FDK-initialisation oracle (Sec. 4.1) against closed forms, analytic
phantoms, library routines and published generator values.  CPU only."""
import os

import numpy as np
import pytest
from scipy import signal, stats
from scipy.spatial import cKDTree

from oracle import fdk
from paper_2405_20693_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_coords(n):
    xs = -1 + (np.arange(n) + 0.5) * 2 / n
    return np.meshgrid(xs, xs, xs, indexing="ij")  # Z, Y, X


def test_ramp_taps_frequency_response():
    """The band-limited ramp's DTFT is |f| (cycles per sample) below Nyquist; with the
    full-circle factor 1/2 it is |f|/2.  Truncating the taps at +-511 leaves a DC
    residue of about sum_{odd n > 511} 1/(pi^2 n^2) ~ 1e-4."""
    c = fdk.ramp_taps(511)
    n = np.arange(-511, 512)
    assert c[511] == 0.125 and c[512] == pytest.approx(-1 / (2 * np.pi ** 2)) and c[513] == 0.0
    for f in (0.0, 0.03, 0.1, 0.25, 0.4, 0.49):
        H = (c * np.cos(2 * np.pi * f * n)).sum()
        assert abs(H - abs(f) / 2) <= 2e-4, (f, H)


def test_filter_matches_fft_convolution():
    """Row filtering = scipy's FFT convolution with the same taps, pre-weighted."""
    g = I.rng(3)
    cam = I.cone_camera(6, 20, pitch=0.05)
    proj = g.standard_normal((2, 6, 20))
    got = fdk.fdk_filter(proj, cam)
    xi, eta = fdk.detector_coords(cam)
    XI, ETA = np.meshgrid(xi, eta)
    wp = proj * cam.L_SD / np.sqrt(cam.L_SD ** 2 + XI ** 2 + ETA ** 2)
    c = fdk.ramp_taps(19)
    ref = np.stack([np.stack([signal.fftconvolve(wp[v, r], c, mode="same") for r in range(6)]) for v in range(2)])
    assert np.abs(got - ref / cam.pitch_u).max() <= 1e-12 * np.abs(ref).max()


def test_backproject_index_mapping_parallel():
    """Parallel beam, one view at theta = 0 (u = (y, -z, L_SO - x)): with voxel centres
    on pixel centres, bilinear interpolation returns the pixel itself, so the
    back-projection is dbeta * F[row of -z, column of y] for every x."""
    cam = I.parallel_camera(8, 8, 0.25)
    views = I.view_table([0.0], 4.0, dtype=np.float64)
    F = I.rng(4).standard_normal((1, 8, 8))
    vol = fdk.fdk_backproject(F, views, cam, I.cube_grid(8), 0.7).reshape(8, 8, 8)
    for z in range(8):
        for y in range(8):
            assert np.allclose(vol[z, y, :], 0.7 * F[0, 7 - z, y], rtol=0, atol=1e-13)


def test_fdk_cone_reconstructs_z_invariant_cylinder():
    """FDK is exact for objects that do not vary along the rotation axis: a unit-density
    cylinder (an ellipsoid with a 30-unit z semi-axis) scanned with 180 cone-beam views
    reconstructs to 1 inside, 0 outside, on every slice within the cone's field of view."""
    cyl = I.Phantom(np.zeros((1, 3)), np.array([[0.5, 0.5, 30.0]]), np.eye(3)[None], np.array([1.0]))
    cam = I.cone_camera(96, 128, pitch=I.CONE_PITCH * 4)
    views = I.view_table(I.even_angles(180), I.CONE_L_SO, dtype=np.float64)
    proj = I.phantom_projections(cyl, views, cam)
    vol = fdk.fdk(proj, views, cam, I.cube_grid(40), 2 * np.pi / 180).reshape(40, 40, 40)
    Z, Y, X = _grid_coords(40)
    r2 = X ** 2 + Y ** 2
    inside = (r2 < 0.4 ** 2) & (np.abs(Z) < 0.5)
    outside = (r2 > 0.6 ** 2) & (r2 < 0.9 ** 2) & (np.abs(Z) < 0.5)
    assert abs(vol[inside].mean() - 1) < 2e-3
    assert np.abs(vol[inside] - 1).max() < 5e-3
    assert np.abs(vol[outside]).max() < 0.03


def test_fbp_parallel_reconstructs_ball():
    """Parallel beam: slice-by-slice filtered back-projection reconstructs any object;
    a unit ball comes back as 1 inside and 0 outside up to sampling."""
    ball = I.Phantom(np.zeros((1, 3)), np.array([[0.5, 0.5, 0.5]]), np.eye(3)[None], np.array([1.0]))
    cam = I.parallel_camera(64, 96, 2.4 / 96)
    views = I.view_table(I.even_angles(180), 4.0, dtype=np.float64)
    vol = fdk.fdk(I.phantom_projections(ball, views, cam), views, cam, I.cube_grid(40),
                  2 * np.pi / 180).reshape(40, 40, 40)
    Z, Y, X = _grid_coords(40)
    R2 = X ** 2 + Y ** 2 + Z ** 2
    assert abs(vol[R2 < 0.4 ** 2].mean() - 1) < 2e-3
    assert np.abs(vol[R2 < 0.4 ** 2] - 1).max() < 1e-2
    assert np.abs(vol[(R2 > 0.6 ** 2) & (R2 < 0.9 ** 2)]).max() < 0.03


def test_splitmix64_published_values():
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if not l.startswith("#")]
    seed = int(lines[0].split()[1])
    want = [int(l) for l in lines[1:]]
    assert [int(x) for x in fdk.splitmix64_stream(seed, len(want))] == want


def test_sample_candidates_is_a_uniform_subset():
    """Exactly M distinct candidates, ascending; all candidates when there are at most
    M; over many seeds every candidate is drawn with probability M / N (chi-square)."""
    g = I.rng(5)
    vol = g.uniform(0, 1, (6, 7, 8))
    cand = np.flatnonzero(vol.ravel() > 0.3)
    idx = fdk.sample_candidates(vol, 0.3, 40, 17)
    assert idx.size == 40 and np.all(np.diff(idx) > 0) and np.isin(idx, cand).all()
    assert np.array_equal(fdk.sample_candidates(vol, 0.3, cand.size + 5, 17), cand)
    assert not np.array_equal(idx, fdk.sample_candidates(vol, 0.3, 40, 18))
    counts = np.zeros(vol.size)
    S = 4000
    for s in range(S):
        counts[fdk.sample_candidates(vol, 0.3, 40, s)] += 1
    assert counts[np.setdiff1d(np.arange(vol.size), cand)].sum() == 0
    exp = S * 40 / cand.size
    chi2 = ((counts[cand] - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2, cand.size - 1) > 1e-3


def test_knn3_matches_kdtree():
    P = I.rng(6).uniform(-1, 1, (700, 3))
    d, _ = cKDTree(P).query(P, k=4)
    assert np.abs(fdk.knn3_mean_distance(P, chunk=128) - d[:, 1:].mean(axis=1)).max() <= 1e-14


def test_init_gaussians_composition():
    """Sec. 4.1: positions = chosen voxel centres, isotropic 3-NN scales, identity
    rotations, rho = k * volume."""
    g = I.rng(7)
    vol = g.uniform(0, 1, (10, 9, 8))
    gd = I.grid_desc((-0.5, -0.4, -0.3), (0.1, 0.1, 0.12), (8, 9, 10))
    mean, scale, quat, rho = fdk.init_gaussians(vol, gd, 0.5, 60, 3, 0.15)
    idx = fdk.sample_candidates(vol, 0.5, 60, 3)
    z, y, x = np.unravel_index(idx, vol.shape)
    assert np.allclose(mean, np.stack([-0.5 + (x + 0.5) * 0.1, -0.4 + (y + 0.5) * 0.1, -0.3 + (z + 0.5) * 0.12], 1))
    d, _ = cKDTree(mean).query(mean, k=4)
    assert np.allclose(scale, np.repeat(d[:, 1:].mean(1)[:, None], 3, 1), rtol=1e-14)
    assert np.array_equal(quat, np.tile([1.0, 0, 0, 0], (60, 1)))
    assert np.allclose(rho, 0.15 * vol.ravel()[idx], rtol=1e-15)
