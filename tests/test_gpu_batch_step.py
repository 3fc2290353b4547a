"""The fused training step (r2g_train_step) in the configurations bench.py times,
against the oracle's composition of the same iteration (Eq. 8): losses, Adam's
first moment after one step from a fresh state ((1 - beta1) times the gradient of
the raw parameters), and the full volume of the batch form.  The Gaussians are
anisotropic and randomly rotated, so every parameter group, the rotations
included, has a non-zero gradient."""
import numpy as np
import pytest
import torch

from gpu_util import assert_grads_close, assert_values_close, host
from oracle import core, losses
from paper_2405_20693_b300 import build, engine, r2g
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def entry_table(rows):
    t = np.zeros((len(rows), 8), np.int32)
    f = t.view(np.float32)
    for j, (v, it, origin) in enumerate(rows):
        t[j, 0], t[j, 1] = v, it
        f[j, 2:5] = origin
    return torch.as_tensor(t, device="cuda")


def check_step_against_oracle(sc, act_before, raw_before, views, meas, cam, patch_gds, label):
    """The step just taken on sc (from a fresh state) against the oracle: projection
    loss of `views` vs `meas`, the summed TV of the patches, and Adam's first moment
    against the oracle's adjoints chained through the activations.

    Gate band through the loss: a pixel where some Gaussian's q lies within 1e-4 Q of
    the gate may hold that Gaussian's e^{-Q/2} rho_hat on the GPU and not in the oracle
    (the image tolerance widens by exactly that), and the loss gradient dL/dI around
    it -- through the 11 x 11 SSIM window and the L1 sign -- then differs for every
    Gaussian that covers the window.  The oracle measures that effect by evaluating
    dL/dI at its image plus and minus the band image and chaining both differences
    through its adjoint; their magnitudes widen each element's tolerance beside the
    pair's own band."""
    Ga = I.GaussianSet(act_before[1], act_before[2], act_before[0], act_before[3])
    img, _, iband = core.render(Ga, views, cam, Q=engine.Q_PIXEL, want_band=True)
    L1, dimg = losses.projection_loss(img, meas, engine.LAMBDA_SSIM)
    prop = [np.zeros_like(x) for x in (Ga.mean, Ga.scale, Ga.quat, Ga.rho)]
    for sgn in (1.0, -1.0):
        _, d2 = losses.projection_loss(img + sgn * iband, meas, engine.LAMBDA_SSIM)
        for acc, gg in zip(prop, core.render_backward(Ga, views, cam, d2 - dimg, Q=engine.Q_PIXEL)):
            acc += np.abs(gg)
    vols, _ = core.voxelize(Ga, patch_gds, engine.Q_VOXEL)
    D = int(patch_gds[0, 6])
    Ltv, dvol = 0.0, []
    for p in range(patch_gds.shape[0]):
        lt, dv = losses.tv3d(vols[p * D ** 3:(p + 1) * D ** 3].reshape(D, D, D), engine.LAMBDA_TV)
        Ltv += lt
        dvol.append(dv.ravel())
    loss = host(sc.loss)
    assert abs(loss[0] - L1) <= 1e-4 * abs(L1), (label, loss[0], L1)
    assert abs(loss[1] - Ltv) <= 1e-4 * abs(Ltv) + 1e-7, (label, loss[1], Ltv)
    gr, br = core.render_backward(Ga, views, cam, dimg, Q=engine.Q_PIXEL, want_band=True)
    gv, bv = core.voxelize_backward(Ga, patch_gds, np.concatenate(dvol), engine.Q_VOXEL, want_band=True)
    sig = 1.0 / (1.0 + np.exp(-raw_before[3].astype(np.float64)))
    chain = {"quat": 1.0, "mean": 1.0, "scale": act_before[2], "rho": sig}
    ref = {"mean": gr[0] + gv[0], "scale": gr[1] + gv[1], "quat": gr[2] + gv[2], "rho": gr[3] + gv[3]}
    band = {"mean": br[0] + bv[0] + prop[0], "scale": br[1] + bv[1] + prop[1], "quat": br[2] + bv[2] + prop[2],
            "rho": br[3] + bv[3] + prop[3]}
    mq, mm, ms, mr = (host(t) / 0.1 for t in sc.state.views_of(sc.state.m))
    for name, got in (("quat", mq), ("mean", mm), ("scale", ms), ("rho", mr)):
        want = ref[name] * chain[name]
        assert np.abs(want).max() > 0, (label, name)  # rotated Gaussians: every group moves
        assert_grads_close(got, want, f"{label} d{name} (raw)", band=band[name] * np.abs(chain[name]))
    return Ga


def test_batch_step_matches_oracle_composition():
    """The batch form (all 5 views of a cone scan in one launch, 3 TV patches at
    device-read origins, the full 64^3 volume) from a fresh state: both losses,
    Adam's first moment and the full volume against the oracle."""
    G = I.uniform_gaussians(4000, 31, 0.01, 0.06, box=0.7)
    ph, _ = I.normalised_phantom(31, 64)
    cam = I.cone_camera(128, 128, pitch=I.CONE_PITCH * 4)
    views = I.view_table(np.deg2rad([7.0, 80.0, 151.0, 222.0, 300.0]), I.CONE_L_SO)
    meas = I.phantom_projections(ph, views, cam, device="cuda").astype(np.float32)
    sc = engine.Scan(G, views, meas, cam, n_out=64, D=16, tile=(16, 16), all_views=True, n_patches=3,
                     full_volume=True)
    act = [host(t) for t in sc.state.views_of(sc.state.act)]
    raw = [host(t) for t in sc.state.views_of(sc.state.raw)]
    origins = np.array([[-0.5, -0.25, 0.0], [0.0, 0.125, -0.375], [-0.25, -0.5, -0.5]], np.float32)
    sc.patch_origins.copy_(torch.as_tensor(origins))
    table = entry_table([(0, 0, (0.0, 0.0, 0.0))])
    r2g.r2g_train_step(sc.job, table.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert not sc.overflowed()
    gds = np.stack([np.asarray(I.grid_desc(o, (2 / 64,) * 3, (16, 16, 16)), np.float32).astype(np.float64)
                    for o in origins])
    Ga = check_step_against_oracle(sc, act, raw, views, meas.astype(np.float64), cam, gds, "batch step")
    ref, _, band = core.voxelize(Ga, np.asarray(I.cube_grid(64), np.float32).astype(np.float64), engine.Q_VOXEL,
                                 want_band=True)
    assert_values_close(host(sc.full_vol), ref, band, "batch step full volume")


def test_one_scan_step_full_size_rotated():
    """The one-scan bench step exactly as timed -- r2g_train_step with 32x32 tiles, the
    cooperative projection + list build, records copied next to the sorted entries,
    programmatic dependent launches -- at full size (512^2 view, 50 views, 32^3 TV
    patch at the 256^3 spacing) on 50,000 anisotropic, randomly rotated Gaussians from
    the bench phantom: losses and Adam's first moment against the oracle."""
    ph, vol = I.normalised_phantom(0, 256)
    G = I.init_from_volume(vol, I.cube_grid(256), 50_000, 5, scale_override=(0.003, 0.03), random_rot=True)
    cam = I.cone_camera(512, 512)
    views = I.view_table(I.even_angles(50), I.CONE_L_SO)
    v = 29
    meas = np.zeros((50, 512, 512), np.float32)
    meas[v] = I.phantom_projections(ph, views[v:v + 1], cam, device="cuda")[0]
    sc = engine.Scan(G, views, meas, cam, n_out=256, D=32)
    assert (sc.rast.opts.tile_w, sc.rast.opts.tile_h) == engine.SCAN_TILE == (32, 32)
    act = [host(t) for t in sc.state.views_of(sc.state.act)]
    raw = [host(t) for t in sc.state.views_of(sc.state.raw)]
    origin = tuple(-1.0 + o * (2.0 / 256) for o in (97, 131, 112))
    table = entry_table([(v, 0, origin)])
    r2g.r2g_train_step(sc.job, table.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert not sc.overflowed()
    gd = np.asarray(I.grid_desc(origin, (2 / 256,) * 3, (32, 32, 32)), np.float32).astype(np.float64)[None]
    check_step_against_oracle(sc, act, raw, views[v:v + 1], meas[v:v + 1].astype(np.float64), cam, gd,
                              "one-scan step")


def test_view_chunked_batch_step_equals_stored():
    """The batch step with view_chunk = 2 (5 views: chunks of 2, 2 and 1, the lists of
    the first two rebuilt in the backward, the earlier chunks' gradients added before
    the fused chain rule + Adam of the last) against the same step storing all views:
    the same losses bit for bit (the forward is deterministic), the same Adam moments
    up to the float atomics' rounding, and the oracle's composition."""
    G = I.uniform_gaussians(4000, 32, 0.01, 0.06, box=0.7)
    ph, _ = I.normalised_phantom(32, 64)
    cam = I.cone_camera(128, 128, pitch=I.CONE_PITCH * 4)
    views = I.view_table(np.deg2rad([3.0, 70.0, 160.0, 230.0, 310.0]), I.CONE_L_SO)
    meas = I.phantom_projections(ph, views, cam, device="cuda").astype(np.float32)
    origins = torch.as_tensor(np.array([[-0.5, -0.25, 0.0], [0.0, 0.125, -0.375]], np.float32))
    table = entry_table([(0, 0, (0.0, 0.0, 0.0))])
    res = []
    for vc in (0, 2):
        sc = engine.Scan(G, views, meas, cam, n_out=64, D=16, tile=(16, 16), all_views=True, n_patches=2,
                         view_chunk=vc)
        act = [host(t) for t in sc.state.views_of(sc.state.act)]
        raw = [host(t) for t in sc.state.views_of(sc.state.raw)]
        sc.patch_origins.copy_(origins)
        r2g.r2g_train_step(sc.job, table.data_ptr(), torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert not sc.overflowed()
        res.append((sc, act, raw))
    (a, _, _), (b, act, raw) = res
    assert np.array_equal(host(a.loss), host(b.loss))
    for x, y in zip(a.state.views_of(a.state.m), b.state.views_of(b.state.m)):
        x, y = host(x), host(y)
        assert np.abs(x - y).max() <= 1e-5 * np.abs(x).max()
    gds = np.stack([np.asarray(I.grid_desc(o, (2 / 64,) * 3, (16, 16, 16)), np.float32).astype(np.float64)
                    for o in origins.numpy()])
    check_step_against_oracle(b, act, raw, views, meas.astype(np.float64), cam, gds, "chunked batch step")
