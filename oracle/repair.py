"""FP64 oracle of the learned repair network (a data-parallel extension of the
method: the paper repairs holes only by interpolation and ROI re-rendering,
Sec. 3.1 Stage 3 and Sec. 3.5; the network, its features and its per-tile gate
are defined here and nowhere in the paper).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and bench.py's
CPU baseline. Plain numpy in float64, written from the definitions below with no
tiling, fusion or reordering:

  features (per affiliated-eye pixel, after the forward warp of Stage 2 and the
  hole classification of Stage 3):
    0-2  the affiliated image after classification: the warped colour, at a hole
         outside the edge strips the method's own fill (gap interpolation, else
         the row/column fill), 0 at a hole inside the strips
    3    inverse depth 1/z of the winner (0 at holes and for background samples)
    4    hole mask (1 where no sample landed)
    5    distance to the nearest hole pixel, min(d, 8) / 8 (Euclidean, pixels)
  network: six 3x3 convolutions (cross-correlation, zero padding, stride 1),
    channels 6 -> 32 -> 32 -> 32 -> 32 -> 32 -> 4, ReLU after the first five;
    output channels 0-2 are a correction added to features 0-2 (the fill),
    channel 3 a per-pixel gate logit
  gate: the mean of channel 3 over a 16x16 tile; the tile uses the network fill
    for its hole pixels when sigmoid(gate) >= tau
  loss: mean over hole pixels of |fill - target| (averaged over RGB) plus
    lam * mean over tiles of the binary cross-entropy of the gate against a
    label supplied by the caller

Weights are W[l] with shape (c_out, 3, 3, c_in) and b[l] with shape (c_out,).
With bf16=True the inputs, weights and every stored activation are rounded to
bfloat16 (round to nearest even) at the points where the GPU stores them, and
the sums stay in float64, so the GPU's FP32 accumulation is compared against
an exact sum of the same bfloat16 operands.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (6, 32, 32, 32, 32, 32, 4)
TILE = 16
DIST_CLAMP = 8


def n_params() -> int:
    return sum(CHANNELS[l + 1] * 9 * CHANNELS[l] + CHANNELS[l + 1] for l in range(6))


def unpack(flat):
    """Canonical flat order: for each layer, W (c_out, 3, 3, c_in) then b (c_out)."""
    flat = np.asarray(flat, np.float64)
    W, b, o = [], [], 0
    for l in range(6):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        W.append(flat[o:o + co * 9 * ci].reshape(co, 3, 3, ci))
        o += co * 9 * ci
        b.append(flat[o:o + co].copy())
        o += co
    assert o == flat.size
    return W, b


def pack(W, b):
    return np.concatenate([np.concatenate([W[l].ravel(), b[l].ravel()]) for l in range(6)])


def round_bf16(x):
    """float64 -> nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def distance_to_hole(hole):
    """min(Euclidean distance to the nearest hole pixel, 8) / 8; 0 on holes, 1
    when no hole lies within 8 pixels. Brute force over the 17x17 window."""
    hole = np.asarray(hole, bool)
    H, W = hole.shape
    best = np.full((H, W), DIST_CLAMP * DIST_CLAMP + 1, np.int64)
    for dy in range(-DIST_CLAMP, DIST_CLAMP + 1):
        for dx in range(-DIST_CLAMP, DIST_CLAMP + 1):
            d2 = dy * dy + dx * dx
            if d2 > DIST_CLAMP * DIST_CLAMP or abs(dy) >= H or abs(dx) >= W:
                continue
            sh = np.zeros((H, W), bool)
            ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
            xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
            sh[yd, xd] = hole[ys, xs]  # sh[y, x] = hole[y + dy, x + dx]
            best = np.where(sh & (d2 < best), d2, best)
    d = np.minimum(np.sqrt(best.astype(np.float64)), DIST_CLAMP)
    return d / DIST_CLAMP


def features(rgb, z_warp, hole):
    """(6, H, W) float64: rgb (3, H, W) the affiliated image after hole
    classification, z_warp (H, W) camera depth of the winner (+inf for a
    background sample), hole (H, W)."""
    hole = np.asarray(hole, bool)
    z = np.asarray(z_warp, np.float64)
    inv = np.where(hole | ~np.isfinite(z) | (z <= 0), 0.0, 1.0 / np.where(z > 0, z, 1.0))
    return np.concatenate([np.asarray(rgb, np.float64), inv[None], hole[None].astype(np.float64),
                           distance_to_hole(hole)[None]], 0)


def conv3x3(x, W, b):
    """y[o, i, j] = b[o] + sum_{dy, dx, c} W[o, dy, dx, c] x[c, i + dy - 1, j + dx - 1]
    with zeros outside the image."""
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((W.shape[0], H, Wd)) + b[:, None, None]
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,chw->ohw", W[:, dy, dx, :], xp[:, dy:dy + H, dx:dx + Wd])
    return y


def forward(x, W, b, bf16=False):
    """Returns (out (4, H, W), activations [x, h1, ..., h5]) in float64."""
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    acts = [r(x)]
    h = acts[0]
    for l in range(6):
        y = conv3x3(h, r(W[l]), b[l])
        if l < 5:
            h = r(np.maximum(y, 0.0))
            acts.append(h)
        else:
            return y, acts
    raise AssertionError


def tile_gate(out_gate, tile=TILE):
    """Mean of the gate channel over each tile (partial tiles average their pixels)."""
    H, W = out_gate.shape
    ty, tx = (H + tile - 1) // tile, (W + tile - 1) // tile
    g = np.zeros((ty, tx))
    for i in range(ty):
        for j in range(tx):
            g[i, j] = out_gate[i * tile:(i + 1) * tile, j * tile:(j + 1) * tile].mean()
    return g


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def loss(out, target, hole, label, lam=1.0, tile=TILE, base=None):
    """L1 of the fill (base + out[:3], base = features 0-2) on hole pixels +
    lam * gate BCE (lam = 1, the weight the training uses); returns (L,
    dL/dout)."""
    hole = np.asarray(hole, bool)
    nh = max(int(hole.sum()), 1)
    fill = out[:3] if base is None else np.asarray(base, np.float64) + out[:3]
    diff = fill - target
    L1 = (np.abs(diff) * hole[None]).sum() / (3.0 * nh)
    g = tile_gate(out[3], tile)
    p = sigmoid(g)
    eps = 1e-12
    bce = -(label * np.log(p + eps) + (1 - label) * np.log(1 - p + eps))
    nt = g.size
    L = L1 + lam * bce.mean()
    dout = np.zeros_like(out)
    dout[:3] = np.sign(diff) * hole[None] / (3.0 * nh)
    dg = lam * (p - label) / nt  # d bce / d logit
    H, Wd = out.shape[1:]
    for i in range(g.shape[0]):
        for j in range(g.shape[1]):
            ys, xs = slice(i * tile, min((i + 1) * tile, H)), slice(j * tile, min((j + 1) * tile, Wd))
            n = (ys.stop - ys.start) * (xs.stop - xs.start)
            dout[3, ys, xs] = dg[i, j] / n
    return L, dout


def conv3x3_backward(x, W, dy):
    """Gradients of conv3x3 with respect to x, W and b."""
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("ohw,chw->oc", dy, xp[:, ky:ky + H, kx:kx + Wd])
            dxp[:, ky:ky + H, kx:kx + Wd] += np.einsum("oc,ohw->chw", W[:, ky, kx, :], dy)
    return dxp[:, 1:-1, 1:-1], dW, dy.sum((1, 2))


def backward(acts, W, dout, bf16=False):
    """Gradients (dW[l], db[l]) of the network for dL/dout, from the stored
    activations of forward(). With bf16=True the gradient entering each layer
    (dL/dy of its output) and the weights its input gradient is formed with are
    rounded to bfloat16, the points where the GPU's tensor-core backward stores
    them as operands (the network computes in BF16 with FP32 accumulation); the
    sums stay in float64."""
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    dW, db = [None] * 6, [None] * 6
    dy = r(dout)
    for l in range(5, -1, -1):
        dx, dW[l], db[l] = conv3x3_backward(acts[l], r(W[l]), dy)
        if l > 0:
            dy = r(dx * (acts[l] > 0))
    return dW, db


def init_weights(seed, scale=1.0):
    """He-normal weights, zero biases (the training start point)."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for l in range(6):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        W.append(rng.normal(0.0, scale * np.sqrt(2.0 / (9 * ci)), (co, 3, 3, ci)))
        b.append(np.zeros(co))
    return W, b


# ---------------------------------------------------------------- FP8 (e4m3) path
# The network's FP8 variant: every layer input x_l[c] is stored as an e4m3 code
# q = e4m3(x / sx[l][c]) with a per-channel scale sx from calibration (the
# largest |x_l[c]| seen by the BF16 network over calibration tiles, mapped to
# 448, the largest finite e4m3 value); the input scale is folded into the weights,
# W'[o, ., ., c] = W[o, ., ., c] sx[l][c], which are stored per output channel as
# e4m3(W' / sw[l][o]) with sw = max |W'[o]| / 448; a layer computes
# y[o] = sw[o] * sum(qW * qx) + b[o] in FP32, then ReLU and the next layer's
# quantisation.
E4M3_MAX = 448.0


def round_e4m3(x):
    """float64 -> nearest e4m3 value (ties to even), saturating at +-448."""
    x = np.asarray(x, np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -9)))
    e = np.maximum(e, -6.0)              # subnormals below 2^-6: spacing 2^-9
    step = 2.0 ** (e - 3)                # 3 mantissa bits
    q = a / step
    r = np.floor(q)
    frac = q - r
    r = np.where((frac > 0.5) | ((frac == 0.5) & (np.mod(r, 2) == 1)), r + 1, r)
    v = np.minimum(r * step, E4M3_MAX)
    return np.sign(x) * np.where(a == 0, 0.0, v)


def activation_maxima(x, W, b):
    """Per-layer, per-channel largest |input| of the BF16 network (the
    calibration statistic), shape (6, 32); unused channels 0."""
    _, acts = forward(x, W, b, bf16=True)
    amax = np.zeros((6, 32))
    for l in range(6):
        a = np.abs(acts[l]).reshape(acts[l].shape[0], -1).max(1)
        amax[l, :a.size] = a
    return amax


def fp8_scales(amax, W):
    """Activation scales sx (6, 32) and output-channel weight scales sw (6, 32)."""
    sx = np.maximum(amax, 1e-30) / E4M3_MAX
    sw = np.zeros((6, 32))
    for l in range(6):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        Wf = W[l] * sx[l, :ci][None, None, None, :]
        m = np.abs(Wf).reshape(co, -1).max(1)
        sw[l, :co] = np.maximum(m, 1e-30) / E4M3_MAX
    return sx, sw


def forward_fp8(x, W, b, sx, sw):
    """FP8 network forward; returns out (4, H, W) (float64, exact sums)."""
    h = round_e4m3(x / sx[0, :6][:, None, None])
    for l in range(6):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        Wf = W[l] * sx[l, :ci][None, None, None, :]
        qW = round_e4m3(Wf / sw[l, :co][:, None, None, None])
        y = conv3x3(h, qW, np.zeros(co)) * sw[l, :co][:, None, None] + b[l][:, None, None]
        if l < 5:
            h = round_e4m3(np.maximum(y, 0.0) / sx[l + 1, :co][:, None, None])
        else:
            return y
    raise AssertionError
