"""The checkpoint file format (host side, no GPU): arrays, counters and the
generator state survive a write and a read."""
import numpy as np

from paper_2405_20693_b300 import engine


def test_checkpoint_file_round_trip(tmp_path):
    g = np.random.Generator(np.random.PCG64(123))
    g.integers(0, 10, 7)  # advance the generator
    M = 37
    r = np.random.default_rng(0)
    ck = {"M": M, "it": 1234, "rng": g.bit_generator.state,
          "raw": r.standard_normal(11 * M).astype(np.float32), "act": r.standard_normal(11 * M).astype(np.float32),
          "m": r.standard_normal(11 * M).astype(np.float32), "v": r.random(11 * M).astype(np.float32),
          "dens_grad": r.random(50).astype(np.float32), "dens_count": np.arange(50, dtype=np.float32)}
    path = str(tmp_path / "ck.npz")
    engine.save_checkpoint(ck, path)
    back = engine.load_checkpoint(path)
    assert set(back) == set(ck)
    assert back["M"] == M and back["it"] == 1234
    for k in ("raw", "act", "m", "v", "dens_grad", "dens_count"):
        assert back[k].dtype == np.float32 and np.array_equal(back[k], ck[k]), k
    engine.save_checkpoint(ck, str(tmp_path / "bare"))  # the suffix is added on both sides
    assert np.array_equal(engine.load_checkpoint(str(tmp_path / "bare"))["raw"], ck["raw"])
    h = np.random.Generator(np.random.PCG64(0))
    h.bit_generator.state = back["rng"]
    assert np.array_equal(h.integers(0, 1 << 30, 16), g.integers(0, 1 << 30, 16))
