"""Seeded input generators: shapes, determinism and value ranges."""
import numpy as np

import workloads as W
from oracle import ilqr


def _golden_alphas():
    import os
    p = os.path.join(os.path.dirname(__file__), "golden", "line_search_alphas.txt")
    return [float(l) for l in open(p) if l.strip() and not l.startswith("#")]


def test_oracle_line_search_set_is_the_papers():
    assert tuple(_golden_alphas()) == ilqr.ALPHAS


def test_shapes_and_determinism():
    for fn, B, N, Nq in ((W.cfg_tiny, 8, 10, 1), (lambda: W.cfg_track(B=64), 64, 20, 1),
                         (lambda: W.cfg_uneven(B=32), 32, 40, 1), (lambda: W.cfg_mem(B=16), 16, 30, 30)):
        a, b = fn(), fn()
        assert a["x0"].shape == (B, 13) and a["Q"].shape == (B, Nq, 13)
        assert a["x_ref"].shape == (B, N, 13)
        for k in ("R", "u_ref", "u_lo", "u_hi"):
            assert a[k].shape == (B, 4)
        for k in ("x0", "Q", "x_ref", "R", "u_ref", "u_lo", "u_hi"):
            np.testing.assert_array_equal(a[k], b[k])


def test_value_ranges():
    t = W.cfg_track(B=512)
    assert np.all((t["Q"] >= 0.1) & (t["Q"] <= 10))
    speed = np.linalg.norm(t["x0"][:, 7:10], axis=1)
    assert speed.max() <= 20 and speed.min() >= 0
    np.testing.assert_allclose(np.linalg.norm(t["x0"][:, 3:7], axis=1), 1.0, atol=1e-12)
    assert np.abs(t["x_ref"][:, :, 0]).max() <= 15.0 + 1e-9
    u = W.cfg_uneven(B=256)
    assert u["horizon"].min() >= 5 and u["horizon"].max() <= 40
    assert np.all((u["u_hi"] >= 8.5 * 0.8 - 1e-12) & (u["u_hi"] <= 8.5 * 1.2 + 1e-12))
    h = W.cfg_tiny()
    np.testing.assert_allclose(h["u_ref"], 0.75 * 9.81 / 4)
