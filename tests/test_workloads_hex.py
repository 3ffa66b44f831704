"""The twisted hex-grid input recipe (workloads.twisted_hex_mesh, hex_problem, paper_hex_box)."""
import numpy as np

import workloads as W


def test_twist_is_a_rotation_about_the_vertical_axis():
    n = 5
    x0, h0 = W.twisted_hex_mesh(n, 7, jitter=0.15, twist=0.0)
    x1, h1 = W.twisted_hex_mesh(n, 7, jitter=0.15, twist=0.7)
    xk, _ = W.jittered_kuhn_mesh(n, 7)
    assert np.array_equal(x0, xk)  # same vertices and jitter draws as the tetrahedral box
    assert np.array_equal(h0, h1)
    assert np.array_equal(x1[:, 2], x0[:, 2])
    r0 = np.hypot(x0[:, 0] - 0.5, x0[:, 1] - 0.5)
    r1 = np.hypot(x1[:, 0] - 0.5, x1[:, 1] - 0.5)
    assert np.allclose(r0, r1, rtol=0, atol=1e-15)
    a0 = np.arctan2(x0[:, 1] - 0.5, x0[:, 0] - 0.5)
    a1 = np.arctan2(x1[:, 1] - 0.5, x1[:, 0] - 0.5)
    turn = np.angle(np.exp(1j * (a1 - a0)))
    keep = r0 > 1e-12
    assert np.allclose(turn[keep], 0.7 * x0[keep, 2], rtol=0, atol=1e-12)


def test_hex_connectivity_and_problem_fields():
    n = 3
    xyz, hexes = W.twisted_hex_mesh(n, 1, jitter=0.0, twist=0.0)
    n1 = n + 1
    assert hexes.shape == (n ** 3, 8) and xyz.shape == (n1 ** 3, 3)
    for c in (0, 5, n ** 3 - 1):
        i, j, k = c % n, (c // n) % n, c // (n * n)
        for v in range(8):
            a, b, cc = v & 1, (v >> 1) & 1, v >> 2
            assert np.allclose(xyz[hexes[c, v]], np.array([i + a, j + b, k + cc]) / n)
    base = W.two_material_box(n=4, G=3, n_polar=2, n_az=4)
    cfg = W.hex_problem(base)
    assert cfg["Q"].shape == (64, 3, 8) and cfg["cell_material"].shape == (64,)
    assert np.array_equal(cfg["cell_material"], base["cell_material"][::6])
    assert np.array_equal(cfg["Q"][:, :, 0], base["Q"][::6, :, 0])
    p = W.paper_hex_box()
    assert p["hexes"].shape[0] == 4096 and p["n_groups"] == 10 and p["n_polar"] * p["n_azimuthal"] == 256
