"""Helpers shared by the GPU parity tests: seeded workloads, device transfer and
the tolerance rules (pixel/voxel max error <= 1e-4 of the oracle's max, widened
by the gate-band magnitude the oracle reports; gradients <= 1e-3 relative)."""
import numpy as np
import torch

from paper_2405_20693_b300 import inputs as I

TOL_VALUE = 1e-4
TOL_GRAD = 1e-3


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def dev_set(G):
    return dev(G.mean), dev(G.scale), dev(G.quat), dev(G.rho)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def assert_values_close(gpu, ref, band, label=""):
    """max |gpu - ref| <= 1e-4 max|ref| at every sample, plus the gate-band magnitude
    (a Gaussian whose q sits within 1e-4 Q of the gate may be counted on one side only)."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    band = np.zeros_like(ref) if band is None else np.asarray(band, dtype=np.float64).ravel()
    scale = np.abs(ref).max()
    err = np.abs(gpu - ref)
    allowed = TOL_VALUE * scale + 1.001 * band
    bad = err > allowed
    assert not bad.any(), (f"{label}: {bad.sum()} samples beyond tolerance; worst excess "
                           f"{(err - allowed).max():.3e} (max ref {scale:.3e})")
    return err.max() / scale, int((band > 0).sum())


def assert_grads_close(gpu, ref, label="", band=None, zero_scale=None, tol=None):
    """Per parameter group: ||g - g_ref||_inf <= 1e-3 ||g_ref||_inf, and per element
    |g - g_ref| <= 1e-3 |g_ref| where |g_ref| >= 1e-2 ||g_ref||_inf (tol: another bound
    than 1e-3, for inputs whose FP32 conditioning is known to need it).  Both are widened by
    the oracle's gate-band bound (the summed |contribution| of pairs whose q is within
    1e-4 Q of the gate, which an FP32 gate may count on the other side).  A group that
    is exactly zero in the oracle (e.g. rotations of isotropic Gaussians) must be
    below 1e-6 zero_scale on the GPU."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    band = np.zeros_like(ref) if band is None else np.asarray(band, dtype=np.float64)
    n = np.abs(ref).max()
    if n == 0:
        assert zero_scale is not None, f"{label}: zero reference"
        assert np.abs(gpu).max() <= 1e-6 * zero_scale, f"{label}: {np.abs(gpu).max():.3e} where 0 expected"
        return 0.0, 0.0
    tol = TOL_GRAD if tol is None else tol
    err = np.abs(gpu - ref)
    rel = (err - band).max() / n
    assert rel <= tol, f"{label}: group error {rel:.3e}"
    big = np.abs(ref) >= 1e-2 * n
    el = ((err - 1.001 * band)[big] / np.abs(ref)[big]).max() if big.any() else 0.0
    assert el <= tol, f"{label}: element error {el:.3e}"
    return rel, el


def config1():
    """2,000 anisotropic Gaussians, parallel beam, 4 views at 0/45/90/135 deg, 64x64 at 2/64."""
    G = I.uniform_gaussians(2000, 0)
    cam = I.parallel_camera(64, 64, 2.0 / 64)
    views = I.view_table(np.deg2rad([0.0, 45.0, 90.0, 135.0]), I.CONE_L_SO)
    return G, cam, views


def cone_small(M=3000, seed=7, H=96, W=112, V=3):
    """A reduced cone-beam scan with the paper's geometry (L_SO 1000 mm, L_SD 1500 mm)
    and a coarser detector that still covers the volume."""
    G = I.uniform_gaussians(M, seed, 0.01, 0.08, box=0.8)
    pitch = I.CONE_PITCH * 512 / max(H, W)
    cam = I.cone_camera(H, W, pitch=pitch)
    cam.off_u = 0.5 * pitch  # exercise a detector offset
    views = I.view_table(np.deg2rad(np.arange(V) * (360.0 / V) + 11.0), I.CONE_L_SO)
    return G, cam, views


def config2():
    """The one-scan workload at full size: 50k Gaussians initialised from the seeded
    256^3 phantom, cone beam 1000/1500 mm, 50 views over 360 deg, 512^2 at 0.8 mm."""
    ph, vol = I.normalised_phantom(0, 256)
    G = I.init_from_volume(vol, I.cube_grid(256), 50_000, 0)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(50), I.CONE_L_SO)
    return G, cam, views, ph, vol


def config3(M=500_000, V=75):
    """Differentiation at scale: 500k Gaussians sampled from the phantom support,
    per-axis scales log-U[0.002, 0.05], random rotations, rho = 0.15 V(p); 75 views."""
    ph, vol = I.normalised_phantom(0, 256)
    G = I.init_from_volume(vol, I.cube_grid(256), M, 3, scale_override=(0.002, 0.05), random_rot=True)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(V), I.CONE_L_SO)
    return G, cam, views, ph, vol
