"""Adaptive density control (Sec. 4.2.3) on the CUDA path: the densify step
against the FP64 oracle, the gradient statistics the fused training step
accumulates, and a training run that densifies on the paper's schedule."""
import numpy as np
import pytest
import torch

from gpu_util import dev, host
from oracle import core, densify as D, losses
from paper_2405_20693_b300 import build, engine, r2g
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    r2g.lib()


def _state(M, seed):
    g = I.rng(seed)
    quat = I.random_quats(g, M)
    mean = g.uniform(-0.5, 0.5, (M, 3))
    sc = np.exp(g.uniform(np.log(0.004), np.log(0.06), (M, 3)))
    rho = g.uniform(0.0, 0.5, M)
    rho[g.random(M) < 0.05] = 1e-7                      # empty: pruned
    act = D.join_state({"quat": quat, "mean": mean, "scale": sc, "rho": rho}).astype(np.float32)
    raw = D.join_state({"quat": quat, "mean": mean, "scale": np.log(sc),
                        "rho": D.inv_softplus(rho)}).astype(np.float32)
    m = g.standard_normal(11 * M).astype(np.float32)
    v = g.uniform(0, 1, 11 * M).astype(np.float32)
    cnt = g.integers(0, 4, M).astype(np.float32)
    avg = np.exp(g.uniform(np.log(1e-6), np.log(1e-3), M))
    # keep every mean at least 1e-3 (relative) away from the threshold: FP32 and FP64
    # then take the same decision
    avg = np.where(np.abs(avg / 5e-5 - 1) < 1e-3, avg * 1.01, avg)
    gsum = (avg * cnt).astype(np.float32)
    return raw, act, m, v, gsum, cnt


@pytest.mark.parametrize("M,cap_extra,seed", [(5000, 10 ** 6, 1), (3000, 40, 2), (257, 0, 3)])
def test_densify_matches_oracle(M, cap_extra, seed):
    """Prune / clone / split of a random state against the oracle: the same count and
    layout, survivors copied exactly (a clone's original with rho / 2), copies with
    zero moments, children means and scales to FP32 rounding.  cap_extra limits the
    new Gaussians (40: a cut inside the candidates; 0: no room at all)."""
    raw, act, m, v, gsum, cnt = _state(M, seed)
    cap = M + cap_extra if cap_extra < 10 ** 6 else 4 * M
    opts = r2g.densify_opts(seed=77)
    outs = [torch.empty(11 * cap, device="cuda") for _ in range(4)]
    m_new = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(r2g.r2g_densify_workspace_size(), dtype=torch.uint8, device="cuda")
    r2g.r2g_densify(M, dev(raw), dev(act), dev(m), dev(v), dev(gsum), dev(cnt), opts, cap, *outs, m_new, ws)
    n = int(m_new.item())
    f32 = lambda x: float(np.float32(x))
    (r2, a2, m2, v2), n_ref = D.densify(raw, act, m, v, M, gsum, cnt, grad_threshold=f32(5e-5),
                                        min_density=f32(1e-5), split_scale=f32(0.02), split_factor=f32(1.6),
                                        seed=77, max_gaussians=cap)
    assert n == n_ref
    kind = D.classify(act, M, gsum, cnt, f32(5e-5), f32(1e-5), f32(0.02))
    assert (kind == 0).any() and (kind == 2).any() and (kind == 3).any()
    got = [host(t[:11 * n]) for t in outs]
    G, R = D.split_state(got[1], n), D.split_state(r2, n)
    Gr, Gm, Gv = D.split_state(got[0], n), D.split_state(got[2], n), D.split_state(got[3], n)
    Sa, Sm, Sv = D.split_state(a2, n), D.split_state(m2, n), D.split_state(v2, n)
    for g in D.GROUPS:
        assert np.array_equal(Gm[g], Sm[g]) and np.array_equal(Gv[g], Sv[g]), g
        assert np.allclose(G[g], Sa[g], rtol=2e-6, atol=2e-6), g
        assert np.allclose(Gr[g], R[g], rtol=2e-5, atol=2e-6), g


def test_train_step_accumulates_position_gradient_statistics():
    """One fused step (view 2, a fixed TV patch) from a fresh state with the
    statistics on: per Gaussian, the sum of |dL/dp^| (NDC) and the count of records
    with a gradient, against the oracle's record gradients of the same dL/dI (its own
    render and loss gradient)."""
    spec = I.ScanSpec(240, 3000, 6, 128, 64)
    G, cam, views, meas, _ = I.make_scan(spec, device="cuda")
    sc = engine.Scan(G, views, meas, cam, n_out=64, D=16)
    sc.enable_adaptive(4 * G.M)
    act = [host(t) for t in sc.state.views_of(sc.state.act)]  # quat, mean, scale, rho
    t = np.zeros((1, 8), np.int32)
    t[0, 0] = 2
    t.view(np.float32)[0, 2:5] = (-0.25, -0.25, -0.25)
    r2g.r2g_train_step(sc.job, torch.as_tensor(t, device="cuda").data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    Ga = I.GaussianSet(act[1], act[2], act[0], act[3])
    img, _ = core.render(Ga, views[2:3], cam, Q=engine.Q_PIXEL)
    _, dimg = losses.projection_loss(img, meas[2:3], engine.LAMBDA_SSIM)
    rg = core.record_grads(Ga, views[2:3], cam, dimg, Q=engine.Q_PIXEL)
    s_ref, c_ref = D.grad_stats(rg, cam)
    s_got, c_got = host(sc.dens_grad[:G.M]), host(sc.dens_count[:G.M])
    assert (c_got != c_ref).sum() <= max(2, G.M // 1000)
    assert np.abs(s_got - s_ref).max() <= 2e-3 * s_ref.max()


def test_adaptive_training_densifies_on_schedule():
    """A scan trained for 1200 iterations with adaptive control from iteration 200
    every 100 (the paper's rule on a compressed schedule): the Gaussian count changes
    at every densification, the batched graph is recaptured, the training stays
    finite, and the result is no worse than without adaptive control."""
    spec = I.ScanSpec(241, 6000, 25, 128, 64)
    G, cam, views, meas, vol = I.make_scan(spec, device="cuda")
    gt = torch.as_tensor(vol.astype(np.float32), device="cuda")
    plain = engine.Scan(G, views, meas, cam, n_out=64, D=16, total_iters=1200, seed=1)
    ac = engine.Scan(G, views, meas, cam, n_out=64, D=16, total_iters=1200, seed=1)
    ac.enable_adaptive(8 * G.M, start=200, stop=1000, every=100)
    bt = engine.BatchTrainer([plain, ac], graph=True)
    v0 = ac.version
    counts = []
    for _ in range(1200):
        bt.round()
        if ac.it % 100 == 0 and 200 <= ac.it <= 1000:
            counts.append(ac.M)
    torch.cuda.synchronize()
    assert len(counts) == 9 and ac.version - v0 == 9
    assert counts[-1] > G.M
    res = []
    for sc in (plain, ac):
        vox = engine.Voxelizer(sc.M, I.cube_grid(64))
        v = vox.forward(*sc.state.params()).view(64, 64, 64)
        assert torch.isfinite(v).all()
        res.append(engine.volume_metrics(v, gt))
    assert res[1]["psnr"] > res[0]["psnr"] - 0.5, (res, counts)
