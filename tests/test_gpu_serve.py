"""The continuous-batching server: requests arriving over time are admitted by
HBM footprint, trained together, retired, and each one's result is the same as
training that scan alone."""
import numpy as np
import pytest
import torch

from paper_2405_20693_b300 import build, engine, r2g, serve
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def specs():
    return [I.ScanSpec(300, 3000, 6, 128, 64), I.ScanSpec(301, 1200, 4, 64, 64), I.ScanSpec(302, 6000, 8, 128, 64),
            I.ScanSpec(303, 2000, 5, 64, 64)]


def alone_volume(spec, iters, D=16):
    G, cam, views, meas, vol = I.make_scan(spec, device="cuda")
    sc = engine.Scan(G, views, meas, cam, n_out=spec.n_out, D=D, seed=spec.seed)
    table = torch.zeros((1, 8), dtype=torch.int32).pin_memory()
    tdev = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    t, f = table.numpy(), table.numpy().view(np.float32)
    for _ in range(iters):
        v, it, origin = sc.next_entry()
        t[0, 0], t[0, 1] = v, it
        f[0, 2:5] = origin
        torch.cuda.current_stream().synchronize()
        r2g.r2g_upload_round(tdev, table, 1, torch.cuda.current_stream())
        r2g.r2g_train_step(sc.job, tdev.data_ptr(), torch.cuda.current_stream())
    vox = engine.Voxelizer(sc.M, I.cube_grid(spec.n_out))
    out = serve.Server.volume(sc, vox).cpu().numpy()
    return out, vol.ravel()


def psnr(v, gt):
    return 10 * np.log10(1.0 / np.mean((np.asarray(v, np.float64) - gt) ** 2))


def test_requests_admitted_trained_and_equal_to_alone():
    reqs = [serve.Request(k, sp, arrival=0.05 * k, max_iters=6 + 2 * k, psnr_target=99.0, check_every=4)
            for k, sp in enumerate(specs())]
    srv = serve.Server(hbm_budget_bytes=64 << 30, D=16, keep_volumes=True)
    res = srv.run(reqs)
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert all(r.reason == "iterations" and r.iters == 6 + 2 * r.rid for r in res)
    assert all(r.finished >= r.admitted >= r.arrival for r in res)
    for r, sp in zip(res, specs()):
        vol_alone, gt = alone_volume(sp, r.iters)
        vol_mix = srv.volumes[r.rid]
        assert np.abs(vol_mix - vol_alone).max() <= 1e-3 * np.abs(vol_alone).max(), r.rid
        assert abs(psnr(vol_mix, gt) - psnr(vol_alone, gt)) <= 0.01, r.rid
    summary = serve.summarize(res, srv.wall)
    assert summary["p99_time_to_volume_s"] >= summary["p50_time_to_volume_s"] > 0


def test_admission_respects_the_hbm_budget():
    sp = specs()
    need = [serve.footprint_estimate(s, 16) for s in sp]
    budget = need[0] + need[2] + 1  # room for requests 0 and 2 together, not a third
    reqs = [serve.Request(k, s, arrival=0.0, max_iters=4, psnr_target=99.0, check_every=4) for k, s in enumerate(sp)]
    srv = serve.Server(hbm_budget_bytes=budget, D=16)
    res = srv.run(reqs)
    assert len(res) == 4
    assert srv.max_active <= 2
    # first come first served: request 1 is admitted before request 2
    adm = {r.rid: r.admitted for r in res}
    assert adm[0] <= adm[1] <= adm[2] <= adm[3]


def test_host_faults_leave_the_other_requests_alone():
    """Faults injected on the host: request 1 is cancelled while resident, request 3
    asks for more than the whole HBM budget and is refused at once, request 2's
    measured projections carry a NaN (its first step's loss is not finite: the step
    leaves its parameters as they were and the server quarantines it).  Requests 0
    and 4 finish as they do with no fault at all (same iterations, volumes within the
    tolerance of the alone-vs-mix check: the float-atomic gradients differ between
    any two runs in their last bits)."""
    sp = specs() + [I.ScanSpec(304, 2500, 5, 64, 64)]
    big = I.ScanSpec(305, 4_000_000, 75, 512, 256)
    budget = sum(serve.footprint_estimate(s, 16) for s in sp) + (1 << 20)
    assert serve.footprint_estimate(big, 16) > budget

    def run(faults):
        reqs = []
        for k, s in enumerate(sp):
            spec = big if (faults and k == 3) else s
            data = None
            if faults and k == 2:
                G, cam, views, meas, vol = I.make_scan(s, device="cuda")
                meas = meas.copy()
                meas[:, 5, 7] = np.nan  # a corrupt detector pixel in every view
                data = (G, cam, views, meas, vol)
            reqs.append(serve.Request(k, spec, arrival=0.0, max_iters=12, psnr_target=99.0, check_every=4, data=data))
        srv = serve.Server(hbm_budget_bytes=budget, D=16, keep_volumes=True)
        res = srv.run(reqs, cancellations=[(0.0, 1)] if faults else ())
        return {r.rid: r for r in res}, srv

    clean, srv_c = run(False)
    faulty, srv_f = run(True)
    assert faulty[1].reason == "cancelled" and faulty[3].reason == "refused" and faulty[3].iters == 0
    assert faulty[2].reason == "numeric" and faulty[2].iters >= 1
    for rid in (0, 4):
        assert faulty[rid].reason == clean[rid].reason == "iterations" and faulty[rid].iters == clean[rid].iters
        a, b = srv_c.volumes[rid], srv_f.volumes[rid]
        assert np.abs(a - b).max() <= 1e-3 * np.abs(a).max(), rid
    s = serve.summarize(list(faulty.values()), srv_f.wall)
    assert s["reasons"]["cancelled"] == 1 and s["reasons"]["refused"] == 1 and s["reasons"]["numeric"] == 1
    assert s["completed"] == 2


def test_nonfinite_loss_leaves_the_state_and_reports_numeric():
    """A training step whose projection loss is NaN (a NaN pixel in the measured view)
    takes no update: parameters and both Adam moments stay bit for bit as they were,
    and the raster workspace's status reads R2G_E_NUMERIC; the next step on a clean
    view updates as usual and reports R2G_OK."""
    G, cam, views, meas, _ = I.make_scan(specs()[0], device="cuda")
    meas = meas.copy()
    meas[2, 10, 11] = np.nan
    sc = engine.Scan(G, views, meas, cam, n_out=64, D=16)
    before = [t.clone() for t in (sc.state.raw, sc.state.act, sc.state.m, sc.state.v)]
    t = np.zeros((2, 8), np.int32)
    t[0, 0], t[1, 0], t[1, 1] = 2, 3, 1
    tab = torch.as_tensor(t, device="cuda")
    r2g.r2g_train_step(sc.job, tab[0].data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert not np.isfinite(sc.loss.cpu().numpy()[0])
    assert r2g.r2g_poll(sc.rast.ws)[0] == r2g.R2G_E_NUMERIC
    assert all(torch.equal(a, b) for a, b in zip(before, (sc.state.raw, sc.state.act, sc.state.m, sc.state.v)))
    r2g.r2g_train_step(sc.job, tab[1].data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.all(np.isfinite(sc.loss.cpu().numpy()))
    assert r2g.r2g_poll(sc.rast.ws)[0] == r2g.R2G_OK
    assert not torch.equal(before[0], sc.state.raw)


def test_footprint_estimate_covers_the_allocation():
    """The admission estimate is at least what building a scan allocates on the device
    (torch.cuda.memory_allocated before and after), and not more than three times it."""
    for s in specs():
        G, cam, views, meas, _ = I.make_scan(s, device="cuda")
        torch.cuda.synchronize()
        a0 = torch.cuda.memory_allocated()
        sc = engine.Scan(G, views, meas, cam, n_out=s.n_out, D=16, seed=s.seed)
        torch.cuda.synchronize()
        used = torch.cuda.memory_allocated() - a0
        est = serve.footprint_estimate(s, 16)
        assert used <= est <= 3 * used, (s, used, est)
        del sc
