"""Checkpoint file of the learned preconditioner's weights (host code, no GPU):
write/read round trip, and rejection of foreign, truncated and mismatched files."""
import numpy as np
import pytest


def test_round_trip(rbo, tmp_path):
    n = rbo.lib.rbo_gnn_param_count()
    th = np.random.default_rng(0).standard_normal(n).astype(np.float32)
    p = tmp_path / "w.bin"
    rbo.gnn_write(p, th, seed=12345678901)
    got, seed = rbo.gnn_read(p)
    assert seed == 12345678901
    assert got.dtype == np.float32 and np.array_equal(got, th)
    assert p.stat().st_size == 20 + 4 * n


def test_rejects_bad_files(rbo, tmp_path):
    n = rbo.lib.rbo_gnn_param_count()
    th = np.zeros(n, dtype=np.float32)
    good = tmp_path / "good.bin"
    rbo.gnn_write(good, th, seed=1)
    raw = good.read_bytes()
    for name, data in [("magic", b"NOTAGNN!" + raw[8:]), ("short", raw[:12]),
                       ("truncated", raw[:-4]), ("long", raw + b"\0\0\0\0")]:
        p = tmp_path / f"{name}.bin"
        p.write_bytes(data)
        with pytest.raises(ValueError):
            rbo.gnn_read(p)
    other = tmp_path / "other.bin"
    rbo.gnn_write(other, np.zeros(n + 1, dtype=np.float32), seed=1)
    with pytest.raises(ValueError):
        rbo.gnn_read(other)
