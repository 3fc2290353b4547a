"""Pins of the adaptive-density-control oracle (Sec. 4.2.3) against closed forms,
distributions and invariants.  CPU only."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import core, densify as D
from paper_2405_20693_b300 import inputs as I


def _state(M, seed=0, rho=(0.2, 1.0), scale=(0.005, 0.05)):
    g = I.rng(seed)
    quat = I.random_quats(g, M)
    mean = g.uniform(-0.5, 0.5, (M, 3))
    sc = np.exp(g.uniform(math.log(scale[0]), math.log(scale[1]), (M, 3)))
    r = g.uniform(*rho, M)
    act = D.join_state({"quat": quat, "mean": mean, "scale": sc, "rho": r})
    raw = D.join_state({"quat": quat, "mean": mean, "scale": np.log(sc), "rho": D.inv_softplus(r)})
    m = g.standard_normal(11 * M)
    v = g.uniform(0, 1, 11 * M)
    return raw, act, m, v


def test_split_offsets_are_standard_normal():
    z = np.concatenate([D.split_normals(7, i, c) for i in range(5000) for c in range(2)])
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3
    u = D.uniforms(3, np.arange(20000))
    assert u.min() > 0 and u.max() < 1 and stats.kstest(u, "uniform").pvalue > 1e-3


def test_split_children_follow_the_gaussian():
    """Children means of one Gaussian over many draws: sample mean p, covariance Sigma."""
    raw, act, m, v = _state(1, 3, scale=(0.02, 0.08))
    A = D.split_state(act, 1)
    kids = []
    for s in range(3000):
        (_, a2, _, _), n = D.densify(raw, act, m, v, 1, [1.0], [1.0], split_scale=0.0, seed=s)
        assert n == 2
        kids.append(D.split_state(a2, 2)["mean"])
    P = np.concatenate(kids)
    Rm = D.rotation(A["quat"][0])
    Sigma = Rm @ np.diag(A["scale"][0] ** 2) @ Rm.T
    assert np.abs(P.mean(0) - A["mean"][0]).max() < 4 * A["scale"][0].max() / math.sqrt(6000)
    assert np.abs(np.cov(P.T) - Sigma).max() < 0.1 * np.abs(Sigma).max()


def test_densify_layout_counts_and_moments():
    """Survivors in order (moments kept), then each clone's copy and each split's two
    children (zero moments); pruned ones gone; densities of originals and copies
    halved; raw and activated values consistent; clones conserve mass."""
    M = 40
    raw, act, m, v = _state(M, 5)
    A = D.split_state(act, M)
    gsum = np.zeros(M)
    cnt = np.ones(M)
    gsum[[3, 7, 11, 20]] = 1e-3                      # densify
    A["rho"][[5, 8]] = 1e-7                           # prune
    act = D.join_state(A)
    raw = D.join_state({**D.split_state(raw, M), "rho": D.inv_softplus(A["rho"])})
    A["scale"][7] = [0.1, 0.01, 0.01]                 # large: split
    A["scale"][20] = [0.03, 0.05, 0.2]
    act = D.join_state(A)
    raw = D.join_state({**D.split_state(raw, M), "scale": np.log(A["scale"])})
    kind = D.classify(act, M, gsum, cnt, 5e-5, 1e-5, 0.06)
    assert list(np.flatnonzero(kind == 0)) == [5, 8]
    assert list(np.flatnonzero(kind == 2)) == [3, 11] and list(np.flatnonzero(kind == 3)) == [7, 20]
    (r2, a2, m2, v2), n = D.densify(raw, act, m, v, M, gsum, cnt, split_scale=0.06, seed=1)
    assert n == M - 2 - 2 + 2 + 4
    S = D.split_state(a2, n)
    Rr = D.split_state(r2, n)
    Mm, Vv = D.split_state(m2, n), D.split_state(v2, n)
    surv = [i for i in range(M) if i not in (5, 8, 7, 20)]
    assert len(surv) == M - 4
    Mo, Vo = D.split_state(m, M), D.split_state(v, M)
    for o, i in enumerate(surv):
        assert np.array_equal(S["mean"][o], A["mean"][i]) and np.array_equal(Mm["mean"][o], Mo["mean"][i])
        assert np.array_equal(Vv["quat"][o], Vo["quat"][i])
        assert S["rho"][o] == pytest.approx(A["rho"][i] / (2 if i in (3, 11) else 1), rel=1e-15)
    tail = slice(M - 4, n)
    for g in D.GROUPS:
        assert not np.any(Mm[g][tail]) and not np.any(Vv[g][tail])
    # copies in the order of their originals: 3 (clone), 7 (two children), 11 (clone), 20 (two children)
    src = [3, 7, 7, 11, 20, 20]
    assert np.allclose(S["rho"][M - 4:], A["rho"][src] / 2)
    assert np.allclose(S["scale"][M - 4:], A["scale"][src] / np.array([1, 1.6, 1.6, 1, 1.6, 1.6])[:, None])
    assert np.allclose(np.exp(Rr["scale"]), S["scale"], rtol=1e-13)
    assert np.allclose(np.log1p(np.exp(Rr["rho"])), S["rho"], rtol=1e-12)
    # clones: original + copy carry the original's mass
    mass = lambda rho, sc: rho * np.prod(sc)
    o3 = surv.index(3)
    assert mass(S["rho"][o3], S["scale"][o3]) + mass(S["rho"][M - 4], S["scale"][M - 4]) == \
        pytest.approx(mass(A["rho"][3], A["scale"][3]), rel=1e-14)


def test_densify_capacity_cap():
    """With room for two more Gaussians only the first two candidates (index order)
    are densified; the others stay as they are."""
    M = 12
    raw, act, m, v = _state(M, 6)
    gsum = np.zeros(M)
    gsum[[1, 4, 6, 9]] = 1.0
    (r2, a2, _, _), n = D.densify(raw, act, m, v, M, gsum, np.ones(M), split_scale=1.0, max_gaussians=M + 2)
    assert n == M + 2
    S, A = D.split_state(a2, n), D.split_state(act, M)
    assert S["rho"][1] == pytest.approx(A["rho"][1] / 2) and S["rho"][4] == pytest.approx(A["rho"][4] / 2)
    assert S["rho"][6] == A["rho"][6] and S["rho"][9] == A["rho"][9]


def test_record_position_gradient_matches_mean_gradient():
    """Parallel beam at theta = 0: p^ = (y, -z), so dL/dp^x is dL/dmean_y of the
    complex-step-pinned adjoint, Gaussian by Gaussian; the densify statistic is the
    norm in normalised device coordinates."""
    G = I.uniform_gaussians(6, 2, 0.03, 0.1, box=0.6).astype(np.float64)
    cam = I.parallel_camera(40, 48, 2.0 / 48)
    views = I.view_table([0.0], 4.0, dtype=np.float64)
    dimg = I.rng(3).standard_normal((1, 40, 48))
    rg = core.record_grads(G, views, cam, dimg, Q=9.0)
    dm, _, _, _ = core.render_backward(G, views, cam, dimg, Q=9.0)
    assert np.allclose(rg[0, :, 1], dm[:, 1], rtol=1e-12, atol=1e-14)
    assert np.allclose(-rg[0, :, 2], dm[:, 2], rtol=1e-12, atol=1e-14)
    s, c = D.grad_stats(rg, cam)
    want = np.hypot(rg[0, :, 1] * cam.pitch_u * 24, rg[0, :, 2] * cam.pitch_v * 20)
    assert np.allclose(s, want) and np.array_equal(c, (np.abs(rg[0]).sum(1) > 0).astype(float))
