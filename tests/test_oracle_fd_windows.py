"""The windowed central differences that check the GPU gradients at full size
(fd_windows.OracleLossFD) against the oracle's adjoint of the whole Eq. 8 loss on a
scan small enough for the oracle to render every view in full: rho, mean, scale and
rotation parameters, Gaussians inside and outside the TV patches, Poisson-noised
projections.  A window that dropped part of the SSIM halo, a mis-scaled L1 or TV
mean, or a patch left out would show here.  CPU only."""
import numpy as np

from fd_windows import OracleLossFD
from oracle import core, losses
from paper_2405_20693_b300 import inputs as I


def test_windowed_differences_equal_the_adjoint_of_the_loss():
    ph, vol = I.normalised_phantom(0, 64)
    G = I.init_from_volume(vol, I.cube_grid(64), 3000, 3, scale_override=(0.01, 0.06),
                           random_rot=True).astype(np.float64)
    cam = I.cone_camera(96, 96, pitch=I.CONE_PITCH * 512 / 96)
    views = I.view_table(I.even_angles(6), I.CONE_L_SO).astype(np.float64)
    meas = I.poisson_noise(I.phantom_projections(ph, views, cam), 3, 1e5)
    origins = np.array([[-0.3, -0.2, -0.1], [0.0, 0.1, -0.4]])
    gds = np.stack([np.asarray(I.grid_desc(o, (2 / 64,) * 3, (16,) * 3), np.float64) for o in origins])
    fd = OracleLossFD(G, views, cam, meas, gds)
    img, _ = core.render(G, views, cam)
    _, dimg = losses.projection_loss(img, meas, 0.25)
    vv, _ = core.voxelize(G, gds)
    dv = np.concatenate([losses.tv3d(vv[p * 4096:(p + 1) * 4096].reshape(16, 16, 16), 0.05)[1].ravel()
                         for p in range(2)])
    gr = core.render_backward(G, views, cam, dimg)
    gv = core.voxelize_backward(G, gds, dv)
    ana = [gr[i] + gv[i] for i in range(4)]  # mean, scale, quat, rho
    inside = [i for i in range(G.M)
              if np.any(np.all((G.mean[i] > origins + 0.03) & (G.mean[i] < origins + 0.5 - 0.03), axis=1))]
    ks = inside[:8] + [int(i) for i in np.random.default_rng(0).choice(G.M, 12, replace=False)]
    rows = []
    for j, k in enumerate(ks):
        kind = (3, 0, 1, 2)[j % 4]
        comp = 0 if kind == 3 else j % 3
        eps = {3: 1e-4 * G.rho[k], 0: 1e-4 * G.scale[k].min(), 1: 1e-4 * G.scale[k, comp], 2: 1e-4}[kind]
        f, kink, band = fd.grad(k, kind, comp, eps)
        a = ana[kind][k] if kind == 3 else ana[kind][k, comp]
        rows.append((kind, f, a, kink + band))
    for kd in range(4):
        sel = [r for r in rows if r[0] == kd]
        gmax = max(abs(r[2]) for r in sel)
        for _, f, a, slack in sel:
            assert abs(f - a) <= 1e-4 * max(abs(a), 0.1 * gmax) + slack, (kd, f, a, slack)
    # the patches took part: some sampled Gaussian's TV term is non-zero
    assert any(fd.tv_terms(k, 3, 0, 1e-4 * G.rho[k])[0] != 0.0 for k in inside[:8])
