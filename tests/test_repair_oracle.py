"""Pins of the FP64 repair-network oracle against facts outside it: SciPy's
correlation and exact distance transform, finite differences, torch's bfloat16
rounding, and closed-form networks."""
import numpy as np
import pytest

from oracle import repair as R

scipy_signal = pytest.importorskip("scipy.signal")
scipy_ndimage = pytest.importorskip("scipy.ndimage")


def test_parameter_count():
    assert R.n_params() == 39908
    W, b = R.init_weights(0)
    assert R.pack(W, b).size == 39908
    W2, b2 = R.unpack(R.pack(W, b))
    assert all(np.array_equal(a, c) for a, c in zip(W, W2))


def test_conv_is_zero_padded_cross_correlation():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 9, 11))
    W = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = R.conv3x3(x, W, b)
    for o in range(2):
        ref = b[o] + sum(scipy_signal.correlate2d(x[c], W[o, :, :, c], mode="same", boundary="fill")
                         for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_distance_to_hole_matches_exact_edt():
    rng = np.random.default_rng(2)
    hole = rng.random((40, 50)) < 0.02
    hole[20, 25] = True
    d = R.distance_to_hole(hole)
    edt = scipy_ndimage.distance_transform_edt(~hole)
    np.testing.assert_allclose(d, np.minimum(edt, 8.0) / 8.0, rtol=0, atol=1e-12)
    assert np.all(d[hole] == 0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-6, 6, 1000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(R.round_bf16(x), ref)


def test_identity_network_passes_a_channel_through():
    # every layer copies channel 0 through its centre tap: out = relu(...relu(x0))
    W = [np.zeros((R.CHANNELS[l + 1], 3, 3, R.CHANNELS[l])) for l in range(6)]
    b = [np.zeros(R.CHANNELS[l + 1]) for l in range(6)]
    for l in range(6):
        W[l][0, 1, 1, 0] = 1.0
    rng = np.random.default_rng(4)
    x = rng.normal(size=(6, 12, 10))
    out, acts = R.forward(x, W, b)
    np.testing.assert_allclose(out[0], np.maximum(x[0], 0.0), rtol=0, atol=1e-15)
    assert np.all(out[1:] == 0)


def test_shifted_tap_translates():
    W = [np.zeros((R.CHANNELS[l + 1], 3, 3, R.CHANNELS[l])) for l in range(6)]
    b = [np.zeros(R.CHANNELS[l + 1]) for l in range(6)]
    for l in range(6):
        W[l][0, 1, 2, 0] = 1.0  # reads x[i, j + 1]
    x = np.zeros((6, 4, 16))
    x[0, 2, 10] = 1.0
    out, _ = R.forward(x, W, b)
    expect = np.zeros((4, 16))
    expect[2, 4] = 1.0  # six one-pixel shifts to the left
    np.testing.assert_array_equal(out[0], expect)


def _net_loss(flat, x, target, hole, label):
    W, b = R.unpack(flat)
    out, _ = R.forward(x, W, b)
    return R.loss(out, target, hole, label, base=x[:3])[0]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    H, Wd = 20, 18
    x = rng.random((6, H, Wd))
    hole = rng.random((H, Wd)) < 0.3
    target = rng.random((3, H, Wd))
    W, b = R.init_weights(6)
    flat = R.pack(W, b)
    label = np.array([[1.0, 0.0], [0.0, 1.0]])
    out, acts = R.forward(x, W, b)
    L, dout = R.loss(out, target, hole, label, base=x[:3])
    dW, db = R.backward(acts, W, dout)
    g = R.pack(dW, db)
    idx = rng.choice(flat.size, 60, replace=False)
    # include biases and the last layer, where the L1 kinks are far from the probe
    idx = np.concatenate([idx, [flat.size - 1, flat.size - 5, 1728 + 3]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (_net_loss(flat + e, x, target, hole, label) - _net_loss(flat - e, x, target, hole, label)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_loss_gate_gradient_closed_form():
    # a single tile, gate channel constant c: dL/dc = lam * (sigmoid(c) - label) spread evenly
    out = np.zeros((4, 16, 16))
    out[3] = 0.7
    L, d = R.loss(out, np.zeros((3, 16, 16)), np.zeros((16, 16), bool), np.array([[1.0]]), lam=0.5)
    p = 1 / (1 + np.exp(-0.7))
    assert abs(L - 0.5 * -np.log(p)) < 1e-12
    np.testing.assert_allclose(d[3], 0.5 * (p - 1.0) / 256, rtol=1e-12)


def test_residual_fill_starts_at_the_base():
    # a zero last layer reproduces the base fill: the L1 term is the base's error
    rng = np.random.default_rng(13)
    x = rng.random((6, 16, 16))
    W, b = R.init_weights(1)
    W[5][:] = 0.0
    b[5][:] = 0.0
    out, _ = R.forward(x, W, b)
    hole = rng.random((16, 16)) < 0.5
    target = rng.random((3, 16, 16))
    L, _ = R.loss(out, target, hole, np.array([[0.5]]), lam=0.0, base=x[:3])
    assert abs(L - (np.abs(x[:3] - target) * hole).sum() / (3 * hole.sum())) < 1e-12


def test_features():
    rgb = np.full((3, 5, 6), 0.25)
    z = np.full((5, 6), 2.0)
    z[0, 0] = np.inf
    hole = np.zeros((5, 6), bool)
    hole[2, 3] = True
    f = R.features(rgb, z, hole)
    assert f.shape == (6, 5, 6)
    assert f[3, 1, 1] == 0.5 and f[3, 0, 0] == 0.0 and f[3, 2, 3] == 0.0
    assert np.all(f[:3] == 0.25) and f[4, 2, 3] == 1.0
    assert abs(f[5, 2, 5] - 2.0 / 8.0) < 1e-15 and abs(f[5, 0, 0] - np.hypot(2, 3) / 8) < 1e-15


def test_e4m3_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    rng = np.random.default_rng(31)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.uniform(-3, 2.5, 4000),
                        [0.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -10, 1.0625, 1.1875, 448.0, -448.0]])
    x = x[np.abs(x) <= 448.0]  # beyond the range torch gives no finite code
    ref = torch.tensor(x, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(R.round_e4m3(x), ref)
    # saturation at the largest finite code
    assert R.round_e4m3(1000.0) == 448.0 and R.round_e4m3(-470.0) == -448.0


def test_fp8_network_with_exact_codes_is_the_fp64_network():
    # weights and inputs that are exact e4m3 codes at unit scales and an exact
    # network: the FP8 path reproduces the float64 one
    W = [np.zeros((R.CHANNELS[l + 1], 3, 3, R.CHANNELS[l])) for l in range(6)]
    b = [np.zeros(R.CHANNELS[l + 1]) for l in range(6)]
    for l in range(6):
        W[l][0, 1, 1, 0] = 1.0
        W[l][1, 0, 1, 0] = 0.5
    x = np.zeros((6, 8, 8))
    x[0] = np.random.default_rng(32).integers(0, 8, (8, 8)) * 0.25
    sx = np.ones((6, 32))
    sw = np.full((6, 32), 1.0 / 448.0 * 448.0)  # unit weight scales
    out8 = R.forward_fp8(x, W, b, sx, sw)
    out, _ = R.forward(x, W, b)
    np.testing.assert_array_equal(out8, out)


def test_bf16_backward_on_exact_operands_is_the_fp64_backward():
    """The BF16 backward only rounds: with weights, input and every gradient that
    enters a layer exactly representable in bfloat16 (small dyadic values, single
    nonzero taps so that no sum needs more than 8 bits), it equals the float64
    backward bit for bit; on general operands it stays within a few bfloat16
    ulps (2^-8) of it."""
    H, Wd = 12, 10
    W = [np.zeros((R.CHANNELS[l + 1], 3, 3, R.CHANNELS[l])) for l in range(6)]
    b = [np.zeros(R.CHANNELS[l + 1]) for l in range(6)]
    for l in range(6):
        W[l][0, 1, 1, 0] = 0.5      # centre tap passes channel 0 on, halved
        W[l][0, 0, 1, 0] = 0.25     # and a quarter of the row above
    x = np.zeros((6, H, Wd))
    x[0, 3:9, 2:8] = 1.0
    out, acts = R.forward(x, W, b, bf16=True)
    dout = np.zeros_like(out)
    dout[0, 6, 5] = 0.125
    dout[3, 4, 4] = -0.5
    g64 = R.pack(*R.backward(acts, W, dout))
    g16 = R.pack(*R.backward(acts, W, dout, bf16=True))
    assert np.array_equal(g64, g16) and np.abs(g64).max() > 0
    rng = np.random.default_rng(8)
    Wr, br = R.init_weights(9)
    xr = rng.random((6, 20, 18))
    out, acts = R.forward(xr, Wr, br, bf16=True)
    dout = rng.normal(0.0, 1.0, out.shape)
    g64 = R.pack(*R.backward(acts, Wr, dout))
    g16 = R.pack(*R.backward(acts, Wr, dout, bf16=True))
    rel = np.linalg.norm(g16 - g64) / np.linalg.norm(g64)
    assert 0.0 < rel <= 2 ** -7, rel
