"""Pins of the FP64 oracle against things other than itself: closed forms,
quadrature, library routines, invariants and complex-step derivatives.  CPU only."""
import math

import numpy as np
import pytest
from scipy import ndimage, stats
from scipy.spatial.transform import Rotation

from oracle import core, losses
from paper_2405_20693_b300 import inputs as I

Q9 = 9.0
Q3 = 11.345


def f64(G):
    return G.astype(np.float64)


def small_set(M=6, seed=3, lo=0.05, hi=0.2, box=0.4):
    return f64(I.uniform_gaussians(M, seed, lo, hi, box=box))


# ----------------------------------------------------------------------------- O2 vs O3


def test_ray_integral_closed_form_matches_quadrature():
    """Eq. 5: the line integral of one Gaussian; O2 closed form vs O3 trapezoid rule."""
    g = np.random.default_rng(11)
    G = small_set(20, 4, 0.02, 0.3, box=0.8)
    for i in range(G.M):
        s = g.uniform(-3, 3, 3)
        w = g.standard_normal(3)
        w /= np.linalg.norm(w)
        # aim the ray near the Gaussian so the integral is not vanishingly small
        s = G.mean[i] - 2.0 * w + 0.3 * G.scale[i].max() * g.standard_normal(3)
        exact, quad = core.ray_pair(G.mean[i], G.scale[i], G.quat[i], G.rho[i], s, w)
        assert exact > 0
        # the closed form subtracts c - b^2/a, both ~ |p - s|^2 / sigma^2 ~ 1e4 here,
        # so FP64 cancellation alone allows ~1e-12 relative
        assert abs(exact - quad) <= 1e-11 * abs(exact)


# ----------------------------------------------------------------------------- O1 vs O2


def test_parallel_beam_o1_equals_exact_integral():
    """Parallel beam, no gate: the splatted 2D Gaussian (Eq. 7) is the exact ray integral."""
    G = small_set(8, 5)
    views = I.view_table(np.deg2rad([0.0, 33.0, 90.0, 211.0]), 4.0, dtype=np.float64)
    cam = I.parallel_camera(40, 36, 2.0 / 36)
    cam.off_v = 0.03
    o1, _ = core.render(G, views, cam, Q=math.inf)
    o2 = core.render_exact(G, views, cam)
    assert np.abs(o1 - o2).max() <= 1e-12 * np.abs(o2).max()


def test_mu_equals_ray_through_mean():
    """mu = sqrt(2 pi |Sigma~| / |Sigma^|) (Eq. 7) makes rho_hat equal the exact integral
    along the ray through the mean, for cone and parallel beams."""
    G = small_set(10, 6, 0.03, 0.25, box=0.8)
    views = I.view_table(np.deg2rad([15.0, 140.0]), 4.0, dtype=np.float64)
    cone = I.Camera(beam=1, H=8, W=8, L_SD=6.0, pitch_u=0.4, pitch_v=0.4, near_plane=0.04)
    par = I.parallel_camera(8, 8, 0.25)
    for cam in (cone, par):
        pr = core.project(G, views, cam)
        for v in range(views.shape[0]):
            Wm = views[v, :9].reshape(3, 3)
            t = views[v, 9:]
            for i in range(G.M):
                if cam.beam == 1:
                    src = -Wm.T @ t
                    s, w = src, G.mean[i] - src
                else:
                    w = Wm[2]
                    s = G.mean[i] - 5.0 * w
                exact, _ = core.ray_pair(G.mean[i], G.scale[i], G.quat[i], G.rho[i], s, w)
                assert pr[v, i, 0] == 1.0
                # |Sigma~| / |Sigma^| is a ratio of determinants of ill-scaled matrices
                # (J stretches by L_SD / u2): FP64 rounding reaches ~1e-12 relative
                assert abs(pr[v, i, 9] - exact) <= 1e-11 * abs(exact)


def _local_affine_errors(jmode):
    G = f64(I.uniform_gaussians(3, 5, 0.1, 0.2, box=0.8))
    views = I.view_table(np.deg2rad([20.0]), 4.0, dtype=np.float64)
    out = []
    for gi in range(G.M):
        Gi = G.subset([gi])
        base = I.Camera(beam=1, H=48, W=48, L_SD=6.0, pitch_u=1, pitch_v=1, near_plane=0.04)
        pr = core.project(Gi, views, base)[0, 0]
        errs = []
        for f in (1.0, 0.5, 0.25, 0.125):
            Gf = I.GaussianSet(Gi.mean, Gi.scale * f, Gi.quat, Gi.rho)
            p = 0.08 * f
            cam = I.Camera(beam=1, H=48, W=48, L_SD=6.0, pitch_u=p, pitch_v=p, off_u=pr[1], off_v=pr[2],
                           near_plane=0.04)
            o1, _ = core.render(Gf, views, cam, Q=math.inf, jmode=jmode)
            o2 = core.render_exact(Gf, views, cam)
            errs.append(np.abs(o1 - o2).max() / np.abs(o2).max())
        out.append(errs)
    return np.array(out)


def test_cone_local_affine_error_is_first_order():
    """Cone beam: the local-affine transform (Eq. 6, App. A) is exact only in the limit of
    small Gaussians.  With the detector grid scaled along with the Gaussian, the
    error against the exact integral halves each time the scale halves."""
    e = _local_affine_errors(jmode=0)
    ratios = e[:, :-1] / e[:, 1:]
    assert np.all(ratios > 1.8) and np.all(ratios < 2.6), ratios
    assert np.all(e[:, -1] < 2.5e-3)


def test_depth_row_jacobian_leaves_a_bias():
    """Reading of App. A ('J as in EWA Eq. 29'): with the 3DGS depth row (0, 0, 1) in
    place of u/|u| the error does not vanish with the scale -- a fixed bias of order
    1/cos(gamma) - 1 remains.  This is a planted mistake; the oracle never uses it."""
    e = _local_affine_errors(jmode=1)
    assert np.all(e[:, -1] > 3e-3)
    assert np.all(e[:, -1] / e[:, -2] > 0.9)


# ----------------------------------------------------------------------------- mass


def test_projected_mass_parallel():
    """Sum_pixels I * pitch^2 = sum_i rho_i (2 pi)^{3/2} sqrt|Sigma_i| (untruncated)."""
    g = I.rng(21)
    M = 12
    mean = g.uniform(-0.25, 0.25, (M, 3))
    mean *= 0.4 / np.maximum(np.linalg.norm(mean, axis=1, keepdims=True), 0.4)
    scale = g.uniform(0.05, 0.09, (M, 3))
    quat = I.random_quats(g, M)
    rho = g.uniform(0.2, 1.0, M)
    G = I.GaussianSet(mean, scale, quat, rho)
    pitch = 2.0 / 96
    cam = I.parallel_camera(96, 96, pitch)
    views = I.view_table(np.deg2rad([0.0, 71.0, 154.0]), 4.0, dtype=np.float64)
    expect = (rho * (2 * np.pi) ** 1.5 * np.prod(scale, axis=1)).sum()
    img, _ = core.render(G, views, cam, Q=math.inf)
    for v in range(3):
        assert abs(img[v].sum() * pitch * pitch - expect) <= 1e-9 * expect
    # with the 3-sigma gate the 2D mass inside q <= 9 is 1 - e^{-9/2}
    img9, _ = core.render(G, views, cam, Q=Q9)
    for v in range(3):
        assert abs(img9[v].sum() * pitch * pitch / expect - (1 - math.exp(-4.5))) <= 1e-3


# ----------------------------------------------------------------------------- scatter == brute force


def test_render_scatter_equals_brute_force():
    G = f64(I.uniform_gaussians(60, 0))
    views = I.view_table(np.deg2rad([0, 45, 90, 135]), 4.0)
    cam = I.parallel_camera(32, 32, 2.0 / 32)
    a, pa = core.render(G, views, cam, Q=Q9)
    b, pb = core.render(G, views, cam, Q=Q9, brute=True)
    assert pa == pb
    assert np.array_equal(a, b)
    cone = I.Camera(beam=1, H=32, W=32, L_SD=6.0, pitch_u=3.0 / 32, pitch_v=3.0 / 32, near_plane=0.04)
    a, pa = core.render(G, views, cone, Q=Q9)
    b, pb = core.render(G, views, cone, Q=Q9, brute=True)
    assert pa == pb
    assert np.array_equal(a, b)


def test_voxelize_scatter_equals_brute_force():
    G = f64(I.uniform_gaussians(50, 1))
    grids = np.stack([I.cube_grid(12), I.grid_desc((-0.3, -0.2, -0.5), (0.05, 0.04, 0.06), (9, 7, 10))])
    a, pa = core.voxelize(G, grids, Q3)
    b, pb = core.voxelize(G, grids, Q3, brute=True)
    assert pa == pb
    assert np.array_equal(a, b)


def test_voxelize_matches_library_density():
    """Eq. 3 / Eq. 4 through library routines: scipy's quaternion rotation and its
    multivariate normal pdf, rho * pdf * (2 pi)^{3/2} sqrt|Sigma|."""
    G = f64(I.uniform_gaussians(7, 2, 0.1, 0.4, box=0.5))
    gd = I.cube_grid(6)
    vol, _ = core.voxelize(G, gd, math.inf)
    vol = vol.reshape(6, 6, 6)
    xs = -1 + (np.arange(6) + 0.5) * (2 / 6)
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    pts = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    ref = np.zeros(pts.shape[0])
    for i in range(G.M):
        w, x, y, z = G.quat[i]
        R = Rotation.from_quat([x, y, z, w]).as_matrix()
        S = R @ np.diag(G.scale[i] ** 2) @ R.T
        pdf = stats.multivariate_normal(mean=G.mean[i], cov=S).pdf(pts)
        ref += G.rho[i] * pdf * (2 * np.pi) ** 1.5 * np.sqrt(np.linalg.det(S))
    assert np.abs(vol.ravel() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_voxel_gate_truncation_bound():
    """Dropping the q > Q3 tails changes a voxel by at most e^{-Q3/2} sum rho."""
    G = f64(I.uniform_gaussians(40, 3))
    gd = I.cube_grid(10)
    vi, _ = core.voxelize(G, gd, math.inf)
    vq, _ = core.voxelize(G, gd, Q3)
    assert np.all(vi >= vq - 1e-15)
    assert np.abs(vi - vq).max() <= math.exp(-Q3 / 2) * G.rho.sum()


# ----------------------------------------------------------------------------- invariants


def test_isotropic_on_axis_is_view_independent():
    """An isotropic Gaussian on the rotation axis gives the same image in every view
    (the density is view-independent, Sec. 4.2.1), for both beams."""
    G = I.GaussianSet(np.array([[0.0, 0.0, 0.05]]), np.full((1, 3), 0.12), np.array([[0.3, -0.2, 0.5, 0.7]]),
                      np.array([0.8]))
    views = I.view_table(np.deg2rad([0, 40, 97, 180, 300]), 4.0, dtype=np.float64)
    for cam in (I.parallel_camera(24, 24, 1.0 / 24),
                I.Camera(beam=1, H=24, W=24, L_SD=6.0, pitch_u=1.5 / 24, pitch_v=1.5 / 24, near_plane=0.04)):
        img, _ = core.render(G, views, cam, Q=Q9)
        for v in range(1, 5):
            assert np.abs(img[v] - img[0]).max() <= 1e-12 * img[0].max()


def test_permutation_invariance():
    """Additive composition (Eq. 5): the order of the Gaussians does not matter."""
    G = f64(I.uniform_gaussians(50, 4))
    views = I.view_table(np.deg2rad([10, 100]), 4.0)
    cam = I.Camera(beam=1, H=24, W=24, L_SD=6.0, pitch_u=3.0 / 24, pitch_v=3.0 / 24, near_plane=0.04)
    a, _ = core.render(G, views, cam, Q=Q9)
    perm = I.rng(5).permutation(G.M)
    b, _ = core.render(G.subset(perm), views, cam, Q=Q9)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_z_rotation_equals_angle_shift():
    """App. A: the gantry rotates about z, so rotating the object by alpha about z and
    the gantry by alpha gives the original image."""
    G = small_set(12, 7, 0.04, 0.2, box=0.6)
    alpha = np.deg2rad(23.0)
    Rz = np.array([[np.cos(alpha), -np.sin(alpha), 0], [np.sin(alpha), np.cos(alpha), 0], [0, 0, 1]])
    qz = np.array([np.cos(alpha / 2), 0, 0, np.sin(alpha / 2)])
    Gr = I.GaussianSet(G.mean @ Rz.T, G.scale, np.stack([_qmul(qz, q) for q in G.quat]), G.rho)
    th = np.deg2rad([5.0, 130.0])
    cam = I.Camera(beam=1, H=20, W=22, L_SD=6.0, pitch_u=3.0 / 22, pitch_v=3.0 / 20, near_plane=0.04)
    a, _ = core.render(G, I.view_table(th, 4.0, dtype=np.float64), cam, Q=math.inf)
    b, _ = core.render(Gr, I.view_table(th + alpha, 4.0, dtype=np.float64), cam, Q=math.inf)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def test_parallel_opposite_views_mirror():
    G = small_set(12, 8)
    cam = I.parallel_camera(20, 26, 2.0 / 26)
    a, _ = core.render(G, I.view_table([0.4], 4.0, dtype=np.float64), cam, Q=math.inf)
    b, _ = core.render(G, I.view_table([0.4 + np.pi], 4.0, dtype=np.float64), cam, Q=math.inf)
    assert np.abs(a[0] - b[0][:, ::-1]).max() <= 1e-12 * np.abs(a).max()


# ----------------------------------------------------------------------------- adjoints


@pytest.mark.parametrize("beam", [0, 1])
def test_render_adjoint_matches_complex_step(beam):
    G = small_set(4, 3)
    views = I.view_table(np.deg2rad([10, 37, 100]), 4.0)
    if beam == 0:
        cam = I.parallel_camera(24, 28, 2.0 / 28)
    else:
        cam = I.Camera(beam=1, H=24, W=28, L_SD=6.0, pitch_u=3.0 / 28, pitch_v=3.0 / 24, off_u=0.05, near_plane=0.04)
    g = np.random.default_rng(1).standard_normal((3, cam.H, cam.W))
    dm, ds, dq, dr = core.render_backward(G, views, cam, g, Q=Q9)
    for kind, arr, nc in ((0, dm, 3), (1, ds, 3), (2, dq, 4), (3, dr[:, None], 1)):
        for i in range(G.M):
            for c in range(nc):
                cs = (core.render_cs(G, views, cam, Q9, kind, i, c) * g).sum()
                assert abs(cs - arr[i, c]) <= 1e-10 * max(abs(cs), 1e-8), (kind, i, c, cs, arr[i, c])


def test_render_adjoint_matches_central_differences():
    """Untruncated so the image is smooth; central differences with step 2e-5."""
    G = small_set(3, 9)
    views = I.view_table(np.deg2rad([30, 120]), 4.0)
    cam = I.Camera(beam=1, H=20, W=20, L_SD=6.0, pitch_u=3.0 / 20, pitch_v=3.0 / 20, near_plane=0.04)
    g = np.random.default_rng(2).standard_normal((2, 20, 20))
    dm, ds, dq, dr = core.render_backward(G, views, cam, g, Q=math.inf)
    for name, grad in (("mean", dm), ("scale", ds), ("quat", dq)):
        for i in range(G.M):
            for c in range(grad.shape[1]):
                arrs = {k: getattr(G, k).copy() for k in ("mean", "scale", "quat", "rho")}
                h = 2e-5 * max(1.0, abs(arrs[name][i, c]))
                arrs[name][i, c] += h
                up, _ = core.render(I.GaussianSet(**arrs), views, cam, Q=math.inf)
                arrs[name][i, c] -= 2 * h
                dn, _ = core.render(I.GaussianSet(**arrs), views, cam, Q=math.inf)
                fd = ((up - dn) * g).sum() / (2 * h)
                assert abs(fd - grad[i, c]) <= 1e-6 * max(abs(grad).max(), 1e-8)


def test_voxelize_adjoint_matches_complex_step():
    G = small_set(4, 10, 0.08, 0.3)
    grids = np.stack([I.cube_grid(10), I.grid_desc((-0.4, -0.3, -0.2), (0.05, 0.05, 0.05), (8, 8, 8))])
    n = 1000 + 512
    g = np.random.default_rng(3).standard_normal(n)
    dm, ds, dq, dr = core.voxelize_backward(G, grids, g, Q3)
    for kind, arr, nc in ((0, dm, 3), (1, ds, 3), (2, dq, 4), (3, dr[:, None], 1)):
        for i in range(G.M):
            for c in range(nc):
                cs = (core.voxelize_cs(G, grids, Q3, kind, i, c) * g).sum()
                assert abs(cs - arr[i, c]) <= 1e-10 * max(abs(cs), 1e-8), (kind, i, c, cs, arr[i, c])


# ----------------------------------------------------------------------------- X-3DGS amplitude (Sec. 4.2.1)


def _cov(scale, quat):
    """Sigma = R S S^T R^T with scipy's rotation of the (w, x, y, z) quaternion."""
    w, x, y, z = quat
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    return R @ np.diag(np.asarray(scale) ** 2) @ R.T


def _aniso(M=5, seed=41):
    """Strongly anisotropic Gaussians (axis ratio up to 5) so mu varies with the view."""
    g = I.rng(seed)
    mean = g.uniform(-0.2, 0.2, (M, 3))
    scale = np.stack([g.uniform(0.02, 0.03, M), g.uniform(0.08, 0.1, M), g.uniform(0.04, 0.1, M)], axis=1)
    return I.GaussianSet(mean, scale, I.random_quats(g, M), g.uniform(0.3, 1.0, M))


def _bump(G, kind, i, comp, h):
    H = I.GaussianSet(*(np.array(a, np.float64) for a in (G.mean, G.scale, G.quat, G.rho)))  # copies
    arr = (H.mean, H.scale, H.quat, H.rho)[kind]
    if kind == 3:
        arr[i] += h
    else:
        arr[i, comp] += h
    return H


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_gated_forms_hold_the_gate_fixed(kind):
    """render_gated / voxelize_gated with the gate set equal to the value set are
    render / voxelize bit for bit, and their central differences in the value set
    (gate fixed) equal the complex-step derivatives, whose gate uses the real part
    and so is fixed by construction."""
    G = small_set(M=8, seed=21, lo=0.05, hi=0.15)
    cam = I.cone_camera(36, 40, pitch=I.CONE_PITCH * 14)
    views = I.view_table(np.deg2rad([20.0, 140.0]), I.CONE_L_SO)
    assert np.array_equal(core.render(G, views, cam)[0], core.render_gated(G, G, views, cam))
    gd = np.asarray(I.grid_desc((-0.45, -0.4, -0.35), (0.05,) * 3, (18, 17, 16)), np.float64)
    assert np.array_equal(core.voxelize(G, gd)[0], core.voxelize_gated(G, G, gd))
    w = np.random.default_rng(22).standard_normal((2, 36, 40))
    wv = np.random.default_rng(23).standard_normal(18 * 17 * 16)
    for i, comp in ((1, 0), (5, kind % 3)):
        h = 1e-5
        fd = ((w * core.render_gated(_bump(G, kind, i, comp, h), G, views, cam)).sum()
              - (w * core.render_gated(_bump(G, kind, i, comp, -h), G, views, cam)).sum()) / (2 * h)
        cs = (w * core.render_cs(G, views, cam, 9.0, kind, i, comp)).sum()
        assert abs(fd - cs) <= 1e-6 * max(abs(cs), 1e-3), (kind, i, fd, cs)
        fv = ((wv * core.voxelize_gated(_bump(G, kind, i, comp, h), G, gd)).sum()
              - (wv * core.voxelize_gated(_bump(G, kind, i, comp, -h), G, gd)).sum()) / (2 * h)
        cv = (wv * core.voxelize_cs(G, gd, Q3, kind, i, comp)).sum()
        assert abs(fv - cv) <= 1e-6 * max(abs(cv), 1e-3), (kind, i, fv, cv)


def test_biased_projected_mass_is_the_2d_gaussian_mass():
    """Parallel beam, no gate: with rho_hat = rho the splat of Gaussian i is an
    unnormalised 2D Gaussian of covariance Sigma^_v (top-left 2x2 of W Sigma W^T), so
    its detector mass is rho 2 pi sqrt|Sigma^_v| -- view-dependent, unlike the 3D
    mass rho (2 pi)^{3/2} sqrt|Sigma| that the rectified splat keeps in every view."""
    G = _aniso()
    pitch = 2.0 / 96
    cam = I.parallel_camera(96, 96, pitch)
    ang = np.deg2rad([0.0, 37.0, 90.0, 151.0])
    views = I.view_table(ang, 4.0, dtype=np.float64)
    masses = []
    for i in range(G.M):
        Gi = G.subset([i])
        img, _ = core.render(Gi, views, cam, Q=math.inf, biased=True)
        S = _cov(G.scale[i], G.quat[i])
        for v in range(len(ang)):
            Wm = views[v, :9].reshape(3, 3)
            Sh = (Wm @ S @ Wm.T)[:2, :2]
            expect = G.rho[i] * 2 * np.pi * np.sqrt(np.linalg.det(Sh))
            got = img[v].sum() * pitch * pitch
            assert abs(got - expect) <= 1e-9 * expect, (i, v, got, expect)
            masses.append(got)
    # the anisotropy makes the biased mass move by more than 10% across views
    m = np.array(masses).reshape(G.M, len(ang))
    assert np.all(m.max(axis=1) / m.min(axis=1) > 1.1)


def test_biased_splat_is_rectified_over_mu():
    """Gaussian by Gaussian the two amplitudes differ by exactly mu_v (Eq. 7): the
    rectified image equals mu_v times the biased one, cone and parallel beam, gated."""
    G = _aniso(4, 43)
    views = I.view_table(np.deg2rad([12.0, 100.0, 222.0]), 4.0, dtype=np.float64)
    cone = I.Camera(beam=1, H=40, W=44, L_SD=6.0, pitch_u=2.5 / 44, pitch_v=2.5 / 40, near_plane=0.04)
    par = I.parallel_camera(40, 44, 2.0 / 44)
    for cam in (cone, par):
        for i in range(G.M):
            Gi = G.subset([i])
            rect, pr = core.render(Gi, views, cam, Q=Q9)
            bias, pb = core.render(Gi, views, cam, Q=Q9, biased=True)
            assert pr == pb
            mu = core.project(Gi, views, cam)[:, 0, 8]
            for v in range(views.shape[0]):
                assert np.abs(rect[v] - mu[v] * bias[v]).max() <= 1e-13 * np.abs(rect[v]).max()


def test_mean_mu_matches_direct_ray_formula():
    """mean_mu = the average over the views that keep the Gaussian of
    sqrt(2 pi / (omega^T Sigma^-1 omega)), omega the unit ray through the mean (the
    view direction for parallel beam, source -> mean for cone beam); a near plane at
    the source distance drops the views in which the Gaussian lies on the source's side."""
    G = _aniso(6, 44)
    ang = np.deg2rad([0.0, 61.0, 133.0, 250.0, 300.0])
    views = I.view_table(ang, 4.0, dtype=np.float64)
    cone = I.Camera(beam=1, H=8, W=8, L_SD=6.0, pitch_u=0.4, pitch_v=0.4, near_plane=4.0)
    par = I.parallel_camera(8, 8, 0.25)
    for cam in (cone, par):
        got = core.mean_mu(G, views, cam)
        n_dropped = 0
        for i in range(G.M):
            Si = np.linalg.inv(_cov(G.scale[i], G.quat[i]))
            vals = []
            for v in range(len(ang)):
                Wm, t = views[v, :9].reshape(3, 3), views[v, 9:]
                if cam.beam == 1:
                    if (Wm @ G.mean[i] + t)[2] <= cam.near_plane:
                        n_dropped += 1
                        continue
                    om = G.mean[i] + Wm.T @ t
                else:
                    om = Wm[2].copy()
                om /= np.linalg.norm(om)
                vals.append(np.sqrt(2 * np.pi / (om @ Si @ om)))
            expect = np.mean(vals) if vals else 0.0
            assert abs(got[i] - expect) <= 1e-11 * expect, (cam.beam, i, got[i], expect)
        if cam.beam == 1:
            assert 0 < n_dropped < G.M * len(ang)


def test_biased_fit_is_view_inconsistent():
    """Sec. 4.2.1's argument on one anisotropic Gaussian: fit the amplitude of each
    view's splat to that view's exact projection by least squares.  Rectified splats
    recover the true density in every view; biased splats recover mu_v rho, which
    changes with the view.  One biased amplitude fitted to all views together is rho
    times the harmonic mean of mu_v (each view's splat energy is proportional to
    sqrt|Sigma^_v|, i.e. to 1 / mu_v), so no single density fits every view."""
    G = _aniso(1, 45)
    pitch = 2.0 / 64
    cam = I.parallel_camera(64, 64, pitch)
    views = I.view_table(np.deg2rad([0.0, 40.0, 85.0, 130.0, 170.0]), 4.0, dtype=np.float64)
    meas = core.render_exact(G, views, cam)
    unit = I.GaussianSet(G.mean, G.scale, G.quat, np.ones(1))
    basis_r, _ = core.render(unit, views, cam, Q=math.inf)
    basis_b, _ = core.render(unit, views, cam, Q=math.inf, biased=True)
    mu = core.project(unit, views, cam)[:, 0, 8]
    rho = G.rho[0]
    fit_r = (basis_r * meas).sum(axis=(1, 2)) / (basis_r ** 2).sum(axis=(1, 2))
    fit_b = (basis_b * meas).sum(axis=(1, 2)) / (basis_b ** 2).sum(axis=(1, 2))
    assert np.abs(fit_r / rho - 1).max() <= 1e-10
    assert np.abs(fit_b / (mu * rho) - 1).max() <= 1e-10
    assert fit_b.max() / fit_b.min() > 1.2
    joint = (basis_b * meas).sum() / (basis_b ** 2).sum()
    assert abs(joint / (rho * len(mu) / (1.0 / mu).sum()) - 1) <= 1e-10


def test_biased_adjoint_matches_complex_step():
    """The biased chain rule (rho_hat = rho: no mu branch) against complex steps."""
    G = small_set(4, 3)
    views = I.view_table(np.deg2rad([10, 37, 100]), 4.0)
    cam = I.Camera(beam=1, H=24, W=28, L_SD=6.0, pitch_u=3.0 / 28, pitch_v=3.0 / 24, off_u=0.05, near_plane=0.04)
    g = np.random.default_rng(4).standard_normal((3, cam.H, cam.W))
    dm, ds, dq, dr = core.render_backward(G, views, cam, g, Q=Q9, biased=True)
    dm_r = core.render_backward(G, views, cam, g, Q=Q9)[0]
    assert np.abs(dm - dm_r).max() > 1e-3 * np.abs(dm_r).max()   # the variants differ
    for kind, arr, nc in ((0, dm, 3), (1, ds, 3), (2, dq, 4), (3, dr[:, None], 1)):
        for i in range(G.M):
            for c in range(nc):
                cs = (core.render_cs(G, views, cam, Q9, kind, i, c, biased=True) * g).sum()
                assert abs(cs - arr[i, c]) <= 1e-10 * max(abs(cs), 1e-8), (kind, i, c, cs, arr[i, c])


# ----------------------------------------------------------------------------- losses


def test_filter_matches_scipy_correlate():
    x = np.random.default_rng(4).standard_normal((23, 31))
    w = losses.gaussian_window()
    assert np.abs(losses.filt(x, w) - ndimage.correlate(x, w, mode="constant", cval=0.0)).max() < 1e-13
    assert abs(w.sum() - 1) < 1e-15


def test_ssim_identities():
    g = np.random.default_rng(5)
    x = g.uniform(0, 1, (20, 24))
    assert abs(losses.ssim(x, x) - 1.0) < 1e-13
    assert np.abs(losses.ssim_grad(x, x)).max() < 1e-13
    y = g.uniform(0, 1, (20, 24))
    assert abs(losses.ssim(x, y) - losses.ssim(y, x)) < 1e-14
    # constant images: interior SSIM = (2ab + C1) / (a^2 + b^2 + C1), C1 = (0.01 L)^2 with L = 1
    a, b = 0.7, 0.2
    S = losses.ssim_parts(np.full((30, 30), a), np.full((30, 30), b), losses.gaussian_window())[-1]
    assert abs(S[15, 15] - (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)) < 1e-12


def test_ssim_of_column_ramps_closed_form():
    """x = a + s c, y = b + t c along the columns c: away from the zero-padded border the
    window's means are a + s c and b + t c (the window is symmetric) and its variances
    and covariance s^2 V, t^2 V, s t V, V the window's second moment; so SSIM has a
    closed form that fixes C1 = (0.01)^2, C2 = (0.03)^2 and the 11-tap, sigma 1.5
    Gaussian window."""
    k = np.arange(11) - 5.0
    w = np.exp(-k * k / (2 * 1.5 ** 2))
    w /= w.sum()
    V = float((w * k * k).sum())
    c = np.arange(40, dtype=np.float64)[None, :].repeat(40, axis=0)
    a, s_, b, t = 0.3, 0.02, 0.5, -0.015
    S = losses.ssim_parts(a + s_ * c, b + t * c, losses.gaussian_window())[-1]
    mx, my = a + s_ * c, b + t * c
    want = ((2 * mx * my + 1e-4) * (2 * s_ * t * V + 9e-4)) / ((mx * mx + my * my + 1e-4) * ((s_ * s_ + t * t) * V + 9e-4))
    assert np.abs(S[10:30, 10:30] - want[10:30, 10:30]).max() < 1e-12


def test_ssim_gradient_matches_complex_step():
    g = np.random.default_rng(6)
    x = g.uniform(0, 1, (16, 18))
    y = g.uniform(0, 1, (16, 18))
    gr = losses.ssim_grad(x, y)
    h = 1e-20
    for (r, c) in [(0, 0), (3, 7), (8, 8), (15, 17), (10, 2)]:
        xc = x.astype(np.complex128)
        xc[r, c] += 1j * h
        cs = losses.ssim(xc, y.astype(np.complex128)).imag / h
        assert abs(cs - gr[r, c]) <= 1e-10 * max(abs(cs), 1e-6)


def test_projection_loss_gradient_matches_central_differences():
    g = np.random.default_rng(7)
    x = g.uniform(0, 1, (2, 14, 15))
    y = g.uniform(0, 1, (2, 14, 15))
    L, G = losses.projection_loss(x, y)
    for idx in [(0, 0, 0), (1, 5, 6), (0, 13, 14), (1, 7, 3)]:
        h = 1e-6
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd = (losses.projection_loss(xp, y)[0] - losses.projection_loss(xm, y)[0]) / (2 * h)
        assert abs(fd - G[idx]) <= 1e-6 * abs(G).max()


def _window_mass_1d(n: int) -> np.ndarray:
    """Share of the 11-tap, sigma 1.5 Gaussian window (normalised to 1) that falls
    inside [0, n) when centred on each of the n positions: the zero padding drops the
    rest."""
    k = np.arange(11) - 5.0
    w = np.exp(-k * k / (2 * 1.5 ** 2))
    w /= w.sum()
    return np.array([sum(w[j] for j in range(11) if 0 <= i + j - 5 < n) for i in range(n)])


@pytest.mark.parametrize("lam", [0.0, 0.25, 1.0])
def test_projection_loss_closed_form_constant_images(lam):
    """Eq. 8's projection term on constant views: render a_v, measurement b_v on an
    H x W detector.  L1 = the mean of |a_v - b_v| over every pixel of the batch (a sum
    would be H W V times larger).  With zero padding the window keeps the share
    m = m_r m_c of its mass at pixel (r, c), so the local means are m a, m b and the
    (co)variances m (1 - m) a^2, m (1 - m) b^2, m (1 - m) a b; SSIM follows in closed
    form, and L = L1 + lambda (1 - mean over views of the mean SSIM).  The gradient
    at lambda = 0 is sign(a_v - b_v) / (V H W) at every pixel."""
    H, W = 13, 18
    a = np.array([0.7, 0.15])
    b = np.array([0.2, 0.4])
    render = np.stack([np.full((H, W), x) for x in a])
    meas = np.stack([np.full((H, W), x) for x in b])
    L, G = losses.projection_loss(render, meas, lam)
    m = np.outer(_window_mass_1d(H), _window_mass_1d(W))
    C1, C2 = 1e-4, 9e-4
    s_mean = 0.0
    for x, y in zip(a, b):
        v = m * (1.0 - m)
        S = ((2 * m * m * x * y + C1) * (2 * v * x * y + C2)) / ((m * m * (x * x + y * y) + C1) * (v * (x * x + y * y) + C2))
        s_mean += S.mean() / len(a)
    want = np.abs(a - b).mean() + lam * (1.0 - s_mean)
    assert abs(L - want) < 1e-12
    if lam == 0.0:
        sg = np.sign(a - b)[:, None, None] * np.ones((2, H, W)) / render.size
        assert np.abs(G - sg).max() < 1e-18


def test_tv_closed_form_and_gradient():
    """TV of the ramp c1 x + c2 y + c3 z is |c1| + |c2| + |c3| (anisotropic, mean over
    differences, unit voxel steps)."""
    D = 9
    z, y, x = np.meshgrid(np.arange(D), np.arange(D), np.arange(D), indexing="ij")
    ramp = 0.3 * x - 0.7 * y + 0.2 * z
    L, _ = losses.tv3d(ramp, lam_tv=1.0)
    assert abs(L - 1.2) < 1e-12
    v = np.random.default_rng(8).standard_normal((6, 7, 5))
    L, G = losses.tv3d(v)
    for idx in [(0, 0, 0), (3, 4, 2), (5, 6, 4)]:
        h = 1e-7
        vp = v.copy()
        vp[idx] += h
        vm = v.copy()
        vm[idx] -= h
        fd = (losses.tv3d(vp)[0] - losses.tv3d(vm)[0]) / (2 * h)
        assert abs(fd - G[idx]) < 1e-7


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g, bias-corrected moments are exactly g and g^2, so
    each step moves a raw parameter by -lr_t * g / (|g| + eps)."""
    M = 5
    g = np.random.default_rng(9)
    raw = {"mean": g.standard_normal((M, 3)), "scale": g.standard_normal((M, 3)),
           "quat": g.standard_normal((M, 4)), "rho": g.standard_normal(M)}
    zero = {k: np.zeros_like(v) for k, v in raw.items()}
    m = {k: np.zeros_like(v) for k, v in raw.items()}
    vv = {k: np.zeros_like(v) for k, v in raw.items()}
    graw = {k: g.standard_normal(v.shape) for k, v in raw.items()}
    for it in range(4):
        act = {"mean": raw["mean"], "quat": raw["quat"], "scale": np.exp(raw["scale"]),
               "rho": losses.softplus(raw["rho"])}
        # activated-parameter gradients whose chain-ruled raw gradient is graw
        gact = {"mean": graw["mean"], "quat": graw["quat"], "scale": graw["scale"] / act["scale"],
                "rho": graw["rho"] * (1 + np.exp(-raw["rho"]))}
        before = {k: v.copy() for k, v in raw.items()}
        losses.adam_step(raw, gact, m, vv, it)
        for k in raw:
            step = -losses.lr_at(k, it) * graw[k] / (np.abs(graw[k]) + 1e-15)
            assert np.abs((raw[k] - before[k]) - step).max() <= 1e-9 * losses.LR0[k]
    assert zero["mean"].sum() == 0
    assert abs(losses.lr_at("mean", 0) - 2e-4) < 1e-18
    assert abs(losses.lr_at("mean", 30000) - 2e-5) < 1e-18


def test_adam_two_step_closed_form():
    """Two steps with different gradients g1, g2 (groups whose activation is the
    identity): unrolling the moment recursions gives the bias-corrected moments
    m^ = (b1 g1 + g2) / (1 + b1) and v^ = (b2 g1^2 + g2^2) / (1 + b2) after step 2,
    which pins both decay rates and the bias correction (a constant gradient does
    not: its corrected moments are g and g^2 for any rates)."""
    b1, b2, eps = 0.9, 0.999, 1e-15
    g = np.random.default_rng(13)
    M = 7
    raw = {"mean": g.standard_normal((M, 3)), "scale": np.zeros((M, 3)), "quat": g.standard_normal((M, 4)),
           "rho": np.zeros(M)}
    m = {k: np.zeros_like(v) for k, v in raw.items()}
    vv = {k: np.zeros_like(v) for k, v in raw.items()}
    g1 = {k: g.standard_normal(raw[k].shape) for k in raw}
    g2 = {k: g.standard_normal(raw[k].shape) for k in raw}
    start = {k: v.copy() for k, v in raw.items()}
    losses.adam_step(raw, g1, m, vv, 0)
    after1 = {k: v.copy() for k, v in raw.items()}
    losses.adam_step(raw, g2, m, vv, 1)
    for k in ("mean", "quat"):
        step1 = -losses.lr_at(k, 0) * g1[k] / (np.abs(g1[k]) + eps)
        mh = (b1 * g1[k] + g2[k]) / (1 + b1)
        vh = (b2 * g1[k] ** 2 + g2[k] ** 2) / (1 + b2)
        step2 = -losses.lr_at(k, 1) * mh / (np.sqrt(vh) + eps)
        assert np.abs((after1[k] - start[k]) - step1).max() <= 1e-12 * losses.LR0[k]
        assert np.abs((raw[k] - after1[k]) - step2).max() <= 1e-12 * losses.LR0[k]
    assert losses.lr_at("mean", 1) == pytest.approx(2e-4 * 0.1 ** (1 / 30000), rel=1e-14)


# ----------------------------------------------------------------------------- phantom + noise


def test_phantom_chords_match_indicator_quadrature():
    ph = I.random_phantom(12, n=6)
    g = np.random.default_rng(10)
    s = g.uniform(-0.2, 0.2, (4, 3)) + np.array([0, 0, -3.0])
    w = g.standard_normal((4, 3)) * 0.1 + np.array([0, 0, 1.0])
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    exact = ph.line_integrals(s, w)
    A = ph.quadric()
    h = 2e-5
    t = np.arange(0, 6.0, h) + h / 2
    for k in range(4):
        pts = s[k] + t[:, None] * w[k]
        dens = np.zeros(t.size)
        for e in range(ph.centre.shape[0]):
            d = pts - ph.centre[e]
            dens += ph.density[e] * (np.einsum("ni,ij,nj->n", d, A[e], d) <= 1.0)
        quad = dens.sum() * h
        assert abs(quad - exact[k]) <= 4 * h * ph.density.sum()


def test_poisson_noise_is_unbiased_in_the_mean():
    proj = np.full((200, 200), 1.3)
    noisy = I.poisson_noise(proj, 3, n0=1e5)
    assert abs(noisy.mean() - 1.3) < 1e-3
    assert 0.002 < noisy.std() < 0.01


def test_view_table_geometry():
    """App. A: W is orthonormal; the source sits at (L_SO cos, L_SO sin, 0)."""
    th = np.deg2rad([0, 30, 200])
    V = I.view_table(th, 7.8125, dtype=np.float64)
    for k in range(3):
        Wm = V[k, :9].reshape(3, 3)
        assert np.abs(Wm @ Wm.T - np.eye(3)).max() < 1e-15
        src = -Wm.T @ V[k, 9:]
        assert np.allclose(src, [7.8125 * np.cos(th[k]), 7.8125 * np.sin(th[k]), 0.0], atol=1e-14)


# ----------------------------------------------------------------------------- FP32 bound replica


def test_fp32_replica_tracks_fp64_projection():
    G = I.uniform_gaussians(300, 12)
    views = I.view_table(np.deg2rad([0, 45, 90, 135]), I.CONE_L_SO)
    cam = I.cone_camera(64, 64, pitch=I.CONE_PITCH * 8)
    of, oi = core.project_f32(G, views, cam)
    pr = core.project(G, views, cam)
    ok = oi[..., 0] == 1
    assert ok.sum() > 0.5 * ok.size
    for k, j in ((0, 1), (1, 2)):
        assert np.abs(of[..., k][ok] - pr[..., j][ok]).max() <= 1e-5 * np.abs(pr[..., j][ok]).max()
    for k, j in ((2, 3), (3, 4), (4, 5)):
        assert np.abs(of[..., k][ok] - pr[..., j][ok]).max() <= 1e-5 * np.abs(pr[..., 3][ok]).max()


@pytest.mark.parametrize("beam", [0, 1])
def test_fp32_tile_bound_covers_the_gate(beam):
    """Every pixel the FP64 gate admits (away from the gate band) lies in the FP32
    pixel box and so in the Gaussian's tile range."""
    G = I.uniform_gaussians(200, 13)
    views = I.view_table(np.deg2rad([0, 45, 90, 135]), I.CONE_L_SO)
    cam = I.parallel_camera(64, 64, 2.0 / 64) if beam == 0 else I.cone_camera(64, 64, pitch=I.CONE_PITCH * 8)
    _, oi = core.project_f32(G, views, cam)
    pr = core.project(G, views, cam)
    xi = (np.arange(cam.W) + 0.5 - cam.W / 2) * cam.pitch_u + cam.off_u
    eta = (np.arange(cam.H) + 0.5 - cam.H / 2) * cam.pitch_v + cam.off_v
    XI, ETA = np.meshgrid(xi, eta)
    for v in range(4):
        for i in range(G.M):
            if pr[v, i, 0] != 1:
                continue
            al, be, ga = pr[v, i, 3:6]
            det = al * ga - be * be
            dx, dy = XI - pr[v, i, 1], ETA - pr[v, i, 2]
            q = (ga * dx * dx - 2 * be * dx * dy + al * dy * dy) / det
            rr, cc = np.nonzero(q <= Q9 * (1 - 1e-4))
            if rr.size == 0:
                continue
            assert oi[v, i, 0] == 1
            c0, c1, r0, r1 = oi[v, i, 1:5]
            assert cc.min() >= c0 and cc.max() <= c1 and rr.min() >= r0 and rr.max() <= r1


# ----------------------------------------------------------------------------- volume metrics (Sec. 5.1)


def test_volume_metrics_closed_forms():
    """3D SSIM = 1 for identical volumes; a volume constant along z has every axial
    slice equal to one image, so its axial SSIM is that image's 2D SSIM; the PSNR of
    a uniform offset e is -20 log10(e)."""
    from oracle import metrics

    g = I.rng(12)
    a = g.uniform(0, 1, (6, 9, 11))
    assert metrics.ssim3d(a, a)["ssim"] == pytest.approx(1.0, abs=1e-12)
    img_a, img_b = g.uniform(0, 1, (9, 11)), g.uniform(0, 1, (9, 11))
    sa = np.repeat(img_a[None], 6, axis=0)
    sb = np.repeat(img_b[None], 6, axis=0)
    assert metrics.ssim3d(sa, sb)["axial"] == pytest.approx(losses.ssim(img_a, img_b), abs=1e-14)
    mse, p = metrics.psnr3d(a, a + 0.01)
    assert mse == pytest.approx(1e-4, rel=1e-9) and p == pytest.approx(40.0, rel=1e-9)


def test_volume_ssim_orientations_permute_with_the_axes():
    """Transposing the volume's axes permutes the three orientation means: swapping
    x and y exchanges coronal and sagittal (an image's SSIM is transpose-invariant);
    swapping z and y exchanges axial and coronal."""
    from oracle import metrics

    g = I.rng(13)
    a = g.uniform(0, 1, (7, 8, 10))
    b = np.clip(a + g.normal(0, 0.2, a.shape), 0, 1)
    m = metrics.ssim3d(a, b)
    mxy = metrics.ssim3d(a.transpose(0, 2, 1), b.transpose(0, 2, 1))
    myz = metrics.ssim3d(a.transpose(1, 0, 2), b.transpose(1, 0, 2))
    assert mxy["axial"] == pytest.approx(m["axial"], abs=1e-14)
    assert mxy["coronal"] == pytest.approx(m["sagittal"], abs=1e-14)
    assert mxy["sagittal"] == pytest.approx(m["coronal"], abs=1e-14)
    assert myz["axial"] == pytest.approx(m["coronal"], abs=1e-14)
    assert myz["coronal"] == pytest.approx(m["axial"], abs=1e-14)
    assert len({round(m[o], 6) for o in ("axial", "coronal", "sagittal")}) == 3


def test_isotropic_tv_closed_form_and_gradient():
    """A linear ramp v = a x + b y + c z: interior voxels have sqrt(a^2 + b^2 + c^2 + eps),
    voxels on the far faces lose that axis' term; a constant volume gives sqrt(eps);
    the hand gradient equals the complex-step derivative (the square root is analytic
    for eps > 0)."""
    D = 5
    a, b, c, eps = 0.3, -0.2, 0.1, 1e-6
    z, y, x = np.meshgrid(np.arange(D), np.arange(D), np.arange(D), indexing="ij")
    vol = a * x + b * y + c * z
    ex = np.where(x < D - 1, a * a, 0) + np.where(y < D - 1, b * b, 0) + np.where(z < D - 1, c * c, 0)
    loss, _ = losses.tv3d_iso(vol, 1.0, eps)
    assert loss == pytest.approx(np.sqrt(ex + eps).mean(), rel=1e-13)
    assert losses.tv3d_iso(np.full((3, 4, 5), 0.7), 1.0, eps)[0] == pytest.approx(np.sqrt(eps), rel=1e-12)
    g = np.random.default_rng(5).uniform(0, 1, (4, 5, 6))
    _, grad = losses.tv3d_iso(g, 0.05, eps)
    h = 1e-30
    for idx in [(0, 0, 0), (1, 2, 3), (3, 4, 5), (2, 0, 5)]:
        gc = g.astype(np.complex128)
        gc[idx] += 1j * h
        cs = losses.tv3d_iso(gc, 0.05, eps)[0].imag / h
        assert abs(cs - grad[idx]) <= 1e-12 * max(1.0, abs(cs)), (idx, cs, grad[idx])


# ----------------------------------------------------------------------------- low-pass dilation (option)


def test_dilation_widens_the_footprint_by_pitch_squared():
    """Parallel beam, untruncated, one isotropic Gaussian of scale s: with dilation d
    (pixels^2) the image is the 2D Gaussian of variance s^2 + d pitch^2 with the
    undilated peak mu rho = sqrt(2 pi) s rho, so the projected mass grows by
    (s^2 + d pitch^2) / s^2 (the dilation breaks Eq. 7's mass invariant)."""
    s, rho, d = 0.06, 0.7, 0.3
    pitch = 2.0 / 80
    cam = I.parallel_camera(80, 80, pitch)
    G = I.GaussianSet(np.array([[0.013, -0.021, 0.0]]), np.full((1, 3), s), np.array([[1.0, 0, 0, 0]]), np.array([rho]))
    views = I.view_table(np.deg2rad([0.0]), 4.0, dtype=np.float64)
    img, _ = core.render(G, views, cam, Q=math.inf, dilation=d)
    pr = core.project(G, views, cam)
    xi = (np.arange(cam.W) + 0.5 - cam.W / 2) * pitch
    XI, ETA = np.meshgrid(xi, xi)
    var = s * s + d * pitch * pitch
    want = math.sqrt(2 * math.pi) * s * rho * np.exp(-((XI - pr[0, 0, 1]) ** 2 + (ETA - pr[0, 0, 2]) ** 2) / (2 * var))
    assert np.abs(img[0] - want).max() <= 1e-12 * want.max()
    mass0 = math.sqrt(2 * math.pi) * s * rho * 2 * math.pi * s * s
    assert abs(img[0].sum() * pitch * pitch / mass0 - var / (s * s)) <= 1e-9
    assert np.array_equal(core.render(G, views, cam, Q=math.inf, dilation=0.0)[0],
                          core.render(G, views, cam, Q=math.inf)[0])


@pytest.mark.parametrize("beam", [0, 1])
def test_dilated_adjoint_matches_complex_step(beam):
    """With a dilation the hand adjoint still equals complex-step derivatives."""
    G = small_set(3, 7)
    views = I.view_table(np.deg2rad([15, 80]), 4.0)
    if beam == 0:
        cam = I.parallel_camera(24, 28, 2.0 / 28)
    else:
        cam = I.Camera(beam=1, H=24, W=28, L_SD=6.0, pitch_u=3.0 / 28, pitch_v=3.0 / 24, off_u=0.05, near_plane=0.04)
    g = np.random.default_rng(9).standard_normal((2, cam.H, cam.W))
    dm, ds, dq, dr = core.render_backward(G, views, cam, g, Q=Q9, dilation=0.3)
    assert np.abs(dm - core.render_backward(G, views, cam, g, Q=Q9)[0]).max() > 1e-4 * np.abs(dm).max()
    for kind, arr, nc in ((0, dm, 3), (1, ds, 3), (2, dq, 4), (3, dr[:, None], 1)):
        for i in range(G.M):
            for c in range(nc):
                cs = (core.render_cs(G, views, cam, Q9, kind, i, c, dilation=0.3) * g).sum()
                assert abs(cs - arr[i, c]) <= 1e-10 * max(abs(cs), 1e-8), (kind, i, c, cs, arr[i, c])


def test_dilated_fp32_tile_bound_covers_the_dilated_gate():
    """The FP32 replica's dilated pixel box holds every pixel the dilated FP64 gate
    admits (away from the gate band), and contains the undilated box."""
    d = 0.3
    G = I.uniform_gaussians(150, 17, 0.01, 0.05)
    views = I.view_table(np.deg2rad([0, 60, 120]), I.CONE_L_SO)
    cam = I.cone_camera(64, 64, pitch=I.CONE_PITCH * 8)
    _, oi = core.project_f32(G, views, cam, dilation=d)
    _, oi0 = core.project_f32(G, views, cam)
    pr = core.project(G, views, cam)
    xi = (np.arange(cam.W) + 0.5 - cam.W / 2) * cam.pitch_u + cam.off_u
    eta = (np.arange(cam.H) + 0.5 - cam.H / 2) * cam.pitch_v + cam.off_v
    XI, ETA = np.meshgrid(xi, eta)
    checked = 0
    for v in range(3):
        for i in range(G.M):
            if pr[v, i, 0] != 1:
                continue
            if oi0[v, i, 0]:
                assert oi[v, i, 0] == 1
                assert oi[v, i, 1] <= oi0[v, i, 1] and oi[v, i, 2] >= oi0[v, i, 2]
                assert oi[v, i, 3] <= oi0[v, i, 3] and oi[v, i, 4] >= oi0[v, i, 4]
            al = pr[v, i, 3] + d * cam.pitch_u ** 2
            be = pr[v, i, 4]
            ga = pr[v, i, 5] + d * cam.pitch_v ** 2
            det = al * ga - be * be
            dx, dy = XI - pr[v, i, 1], ETA - pr[v, i, 2]
            q = (ga * dx * dx - 2 * be * dx * dy + al * dy * dy) / det
            rr, cc = np.nonzero(q <= Q9 * (1 - 1e-4))
            if rr.size == 0:
                continue
            checked += 1
            assert oi[v, i, 0] == 1
            c0, c1, r0, r1 = oi[v, i, 1:5]
            assert cc.min() >= c0 and cc.max() <= c1 and rr.min() >= r0 and rr.max() <= r1
    assert checked > 100
