"""Differentiation at scale: 500k anisotropic, rotated Gaussians, all 75 cone-beam
views of 512^2 in one launch against Poisson-noised projections (1e5 photons per
ray), 8 random 32^3 TV patches.  The gradient of the whole Eq. 8 loss (L1 + 0.25
D-SSIM over the 75 views, plus 0.05 TV over the patches) is taken on the GPU twice
-- through the torch.autograd bridge (engine.rasterize / projection_loss / voxelize
/ tv3d) and by the fused training step in the tile shapes the benchmark chooses
among -- and compared, for 64 seeded parameters across rho, mean, scale and
rotation, with central finite differences of the oracle's FP64 loss.

The oracle never renders the 75 full views (1.4e10 pairs): a parameter of Gaussian
k changes the image only inside its pixel box in each view and the SSIM map only
within 5 pixels of it, so each view is rendered on a window of the box widened by
10 pixels (every Gaussian whose box meets the window, the whole set at the window's
pixels), and the loss change is summed there.  The gate of Gaussian k is held at the
unperturbed parameters (core.render_gated), as the adjoint's is.  The step is
relative (1e-3 of the Gaussian's smallest scale for a mean, of the value for a scale
or density, 1e-3 for a unit-quaternion component), so the truncation error is
negligible; the tolerance is the gradient tolerance (1e-3 relative, floored at 1e-2
of the group's largest), widened by two computed bounds: the kinks of |.| in L1 and
TV that a difference can straddle, and the gate band (pixels within 1e-4 Q of
Gaussian k's gate, where an FP32 gate may decide the other way)."""
import numpy as np
import pytest
import torch

from fd_windows import OracleLossFD
from gpu_util import assert_values_close, config3, dev, dev_set, host
from oracle import core, losses
from paper_2405_20693_b300 import build, engine, r2g
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu

N_PARAMS = 64
EPS = 1e-3
Q = engine.Q_PIXEL
Q3 = engine.Q_VOXEL
D = 32
NP = 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.fixture(scope="module")
def scale_fd():
    G, cam, views, ph, _ = config3()
    clean = I.phantom_projections(ph, views, cam, device="cuda")
    meas = I.poisson_noise(clean, 3, 1e5).astype(np.float32)
    g = I.rng(7)
    offs = g.integers(0, 256 - D + 1, (NP, 3))
    origins = (-1.0 + offs * (2.0 / 256)).astype(np.float32)
    patch_gds = np.stack([np.asarray(I.grid_desc(o, (2 / 256,) * 3, (D,) * 3), np.float32).astype(np.float64)
                          for o in origins])
    Gd = G.astype(np.float64)
    # 64 parameters (seed 4): kinds cycle rho, mean, scale, quat; 16 of the Gaussians lie
    # in a TV patch so that the voxelizer's adjoint takes part
    gs = I.rng(4)
    inside = np.flatnonzero(np.all([(G.mean[:, a] > origins[:, a].min()) & (G.mean[:, a] < origins[:, a].max() + D / 128)
                                    for a in range(3)], axis=0))
    in_patch = []
    for i in gs.permutation(inside):
        lo = origins + 0.02
        hi = origins + D * 2 / 256 - 0.02
        if np.any(np.all((G.mean[i] > lo) & (G.mean[i] < hi), axis=1)):
            in_patch.append(int(i))
        if len(in_patch) == 16:
            break
    rest = [int(i) for i in gs.choice(G.M, N_PARAMS - len(in_patch), replace=False)]
    ks = in_patch + rest
    params = []
    for j, k in enumerate(ks):
        kind = (3, 0, 1, 2)[j % 4]
        comp = 0 if kind == 3 else int(gs.integers(0, 4 if kind == 2 else 3))
        if kind == 3:
            eps = EPS * float(Gd.rho[k])
        elif kind == 0:
            eps = EPS * float(Gd.scale[k].min())
        elif kind == 1:
            eps = EPS * float(Gd.scale[k, comp])
        else:
            eps = EPS
        params.append((k, kind, comp, eps))
    fd = OracleLossFD(Gd, views.astype(np.float64), cam, meas.astype(np.float64), patch_gds)
    ref = [fd.grad(k, kind, comp, eps) for (k, kind, comp, eps) in params]
    return dict(G=G, cam=cam, views=views, meas=meas, origins=origins, patch_gds=patch_gds, params=params, ref=ref,
                windows=fd.windows_checked)


def check_against_fd(scale_fd, grads, label):
    """grads: (dmean, dscale, dquat, drho) host arrays of the activated parameters."""
    params, ref = scale_fd["params"], scale_fd["ref"]
    got = np.array([grads[kind][k] if kind == 3 else grads[kind][k, comp] for (k, kind, comp, _) in params])
    fd = np.array([r[0] for r in ref])
    slack = np.array([r[1] + r[2] for r in ref])
    kinds = np.array([p[1] for p in params])
    assert np.count_nonzero(fd) >= N_PARAMS - 4, f"{label}: too many zero references"
    for kd in range(4):
        sel = kinds == kd
        floor = 1e-2 * np.abs(fd[sel]).max()
        tol = 1e-3 * np.maximum(np.abs(fd[sel]), floor) + slack[sel]
        err = np.abs(got[sel] - fd[sel])
        bad = err > tol
        assert not bad.any(), (f"{label} kind {kd}: {bad.sum()} of {sel.sum()} beyond tolerance; worst "
                               f"{(err - tol).max():.3e}, fd {fd[sel][bad][:4]}, gpu {got[sel][bad][:4]}")
    return np.abs(got - fd).max()


def test_autograd_bridge_gradient_matches_finite_differences(scale_fd):
    """Through torch.autograd: rasterize all 75 views (one launch), Eq. 8's projection
    loss against the noisy projections, voxelize the 8 patches, TV; backward."""
    G, cam, views, meas = scale_fd["G"], scale_fd["cam"], scale_fd["views"], scale_fd["meas"]
    mean, scale, quat, rho = (t.requires_grad_(True) for t in dev_set(G))
    rast = engine.Rasterizer(G.M, views.shape[0], cam, tile=(16, 16))
    img = engine.rasterize(mean, scale, quat, rho, dev(views), rast)
    lp = engine.projection_loss(img, dev(meas))
    vox = engine.Voxelizer(G.M, scale_fd["patch_gds"])
    vol = engine.voxelize(mean, scale, quat, rho, vox)
    lt = engine.tv3d(vol, NP, D)
    (lp + lt).backward()
    torch.cuda.synchronize()
    # the forward at full size, on the windows the oracle rendered
    img_h = host(img.detach())
    for v, (c0, c1, r0, r1), ref, band in scale_fd["windows"]:
        assert_values_close(img_h[v, r0:r1 + 1, c0:c1 + 1], ref, band, f"view {v} window")
    grads = [host(t.grad) for t in (mean, scale, quat, rho)]
    check_against_fd(scale_fd, grads, "autograd bridge")


@pytest.mark.parametrize("tile", [(16, 16), (32, 32)])
def test_fused_scale_step_gradient_matches_finite_differences(scale_fd, tile):
    """The benchmark's step (the batch form of r2g_train_step: all 75 views, 8 patch
    origins read on the device, the full 256^3 volume) from a fresh state: Adam's
    first moment after it is 0.1 times the raw-parameter gradient; chained back to
    the activated parameters it must match the finite differences."""
    G, cam, views, meas = scale_fd["G"], scale_fd["cam"], scale_fd["views"], scale_fd["meas"]
    sc = engine.Scan(G, views, meas, cam, n_out=256, D=D, tile=tile, all_views=True, n_patches=NP,
                     full_volume=True, headroom=1.25)
    act = [host(t) for t in sc.state.views_of(sc.state.act)]
    raw = [host(t) for t in sc.state.views_of(sc.state.raw)]
    sc.patch_origins.copy_(torch.as_tensor(scale_fd["origins"]))
    t = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    r2g.r2g_train_step(sc.job, t.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert not sc.overflowed()
    img_h = host(sc.image)
    for v, (c0, c1, r0, r1), ref, band in scale_fd["windows"]:
        assert_values_close(img_h[v, r0:r1 + 1, c0:c1 + 1], ref, band, f"{tile} view {v} window")
    mq, mm, ms, mr = (host(x) / 0.1 for x in sc.state.views_of(sc.state.m))
    sig = 1.0 / (1.0 + np.exp(-raw[3]))
    grads = [mm, ms / act[2], mq, mr / sig]
    check_against_fd(scale_fd, grads, f"fused step {tile}")
