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
