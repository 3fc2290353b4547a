"""Checkpoint / resume of a training scan: a snapshot taken between iterations and
put back into a freshly built scan continues the run -- the next iteration's losses
bit for bit (the forward, the losses and the list order are deterministic), the
later ones within the drift of the gradient's float-atomic sums."""
import numpy as np
import pytest
import torch

from paper_2405_20693_b300 import build, engine, r2g
from paper_2405_20693_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _scan_inputs():
    spec = I.ScanSpec(311, 3000, 8, 128, 64)
    G, cam, views, meas, _ = I.make_scan(spec, device="cuda")
    return G, cam, views, meas


def _rounds(sc, n, graph):
    bt = engine.BatchTrainer([sc], graph=graph)
    out = []
    for _ in range(n):
        bt.round()
        torch.cuda.synchronize()
        out.append(sc.loss.cpu().numpy().copy())
    return out


def _state_equals(sc, ck):
    s = sc.state
    n = 11 * ck["M"]
    return all(np.array_equal(t[:n].cpu().numpy(), ck[k]) for k, t in (("raw", s.raw), ("act", s.act),
                                                                       ("m", s.m), ("v", s.v)))


def test_resume_from_a_file_continues_the_run(tmp_path):
    G, cam, views, meas = _scan_inputs()
    a = engine.Scan(G, views, meas, cam, n_out=64, D=16, seed=5)
    _rounds(a, 6, graph=False)
    ck = a.checkpoint()
    assert ck["it"] == 6 and ck["M"] == G.M
    path = str(tmp_path / "scan.npz")
    engine.save_checkpoint(ck, path)
    later = _rounds(a, 4, graph=False)
    b = engine.Scan(G, views, meas, cam, n_out=64, D=16, seed=99)  # another generator: the snapshot's wins
    b.restore(engine.load_checkpoint(path))
    assert b.it == 6 and _state_equals(b, ck)
    resumed = _rounds(b, 4, graph=True)
    assert np.array_equal(resumed[0], later[0])  # the same view, patch, state: the same losses
    for x, y in zip(resumed[1:], later[1:]):
        assert np.all(np.abs(x - y) <= 1e-4 * np.abs(y)), (x, y)
    assert b.it == a.it == 10


def test_resume_after_densification():
    """A snapshot taken after adaptive density control changed the Gaussian count is
    restored into a scan built with the initial count: the count, the statistics and
    the state follow the snapshot, the workspaces are re-sized, and the next round's
    losses are the original run's."""
    G, cam, views, meas = _scan_inputs()

    def make():
        sc = engine.Scan(G, views, meas, cam, n_out=64, D=16, seed=7)
        # a threshold every gradient passes: the densification steps change the count
        sc.enable_adaptive(max_gaussians=6000, opts=r2g.densify_opts(grad_threshold=1e-9), start=2, stop=6, every=2)
        return sc

    a = make()
    _rounds(a, 5, graph=False)
    ck = a.checkpoint()
    assert ck["M"] != G.M and "dens_grad" in ck
    nxt = _rounds(a, 1, graph=False)
    b = make()
    b.restore(ck)
    assert b.M == ck["M"] and b.state.M == ck["M"] and _state_equals(b, ck)
    assert np.array_equal(b.dens_grad.cpu().numpy(), ck["dens_grad"])
    assert not b.overflowed()
    assert np.array_equal(_rounds(b, 1, graph=False)[0], nxt[0])


def test_restore_rejects_a_mismatched_snapshot():
    G, cam, views, meas = _scan_inputs()
    sc = engine.Scan(G, views, meas, cam, n_out=64, D=16)
    ck = sc.checkpoint()
    ck["raw"] = ck["raw"][:-1]
    with pytest.raises(ValueError):
        sc.restore(ck)
