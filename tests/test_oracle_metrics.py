"""Pins of the FP64 SSIM oracle against facts outside it: the identity, a
brute-force window sum with explicit loops, constant images in closed form and
symmetry."""
import numpy as np
import pytest

pytest.importorskip("scipy")
from oracle import metrics as M  # noqa: E402


def test_window_is_a_normalised_gaussian():
    w = M.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    # separable: rank one; centre over corner = exp(2 * 25 / (2 sigma^2))
    assert abs(w[5, 5] / w[0, 0] - np.exp(50.0 / (2 * 1.5 ** 2))) < 1e-9 * w[5, 5] / w[0, 0]
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])


def test_identical_images_give_one():
    rng = np.random.default_rng(1)
    x = rng.random((3, 40, 37))
    assert abs(M.ssim(x, x) - 1.0) < 1e-12


def test_brute_force_window_sums():
    # explicit 11x11 sums with zero padding, no convolution routine
    rng = np.random.default_rng(2)
    H, W = 9, 14  # smaller than the window in one direction
    x, y = rng.random((H, W)), rng.random((H, W))
    w = M.gaussian_window()
    ref = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            s = {"x": 0.0, "y": 0.0, "xx": 0.0, "yy": 0.0, "xy": 0.0}
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        g = w[di + 5, dj + 5]
                        s["x"] += g * x[ii, jj]
                        s["y"] += g * y[ii, jj]
                        s["xx"] += g * x[ii, jj] ** 2
                        s["yy"] += g * y[ii, jj] ** 2
                        s["xy"] += g * x[ii, jj] * y[ii, jj]
            mx, my = s["x"], s["y"]
            vx, vy, cxy = s["xx"] - mx * mx, s["yy"] - my * my, s["xy"] - mx * my
            ref[i, j] = ((2 * mx * my + M.C1) * (2 * cxy + M.C2)) / ((mx * mx + my * my + M.C1) * (vx + vy + M.C2))
    np.testing.assert_allclose(M.ssim_map(x, y), ref, rtol=0, atol=1e-12)


def test_constant_images_closed_form():
    # away from the zero-padded border the local means are the constants and
    # every variance vanishes: SSIM = (2pq + C1) / (p^2 + q^2 + C1)
    p, q = 0.3, 0.7
    m = M.ssim_map(np.full((30, 30), p), np.full((30, 30), q))
    expect = (2 * p * q + M.C1) / (p * p + q * q + M.C1)
    np.testing.assert_allclose(m[5:-5, 5:-5], expect, rtol=1e-12)


def test_symmetric_and_lowered_by_noise():
    rng = np.random.default_rng(3)
    x = rng.random((3, 32, 32))
    n1 = x + 0.02 * rng.standard_normal(x.shape)
    n2 = x + 0.1 * rng.standard_normal(x.shape)
    assert abs(M.ssim(x, n1) - M.ssim(n1, x)) < 1e-14
    assert 1.0 > M.ssim(x, n1) > M.ssim(x, n2)
