"""The learned repair network on the GPU (tcgen05 forward and backward, AdamW)
against the FP64 oracle in oracle/repair.py.

Tolerances: the oracle rounds inputs, weights and stored activations to
bfloat16 at the points where the GPU stores them and sums in float64; the GPU
sums the same bfloat16 products in FP32. A stored activation can then land on
the other side of a bfloat16 rounding boundary (relative step 2^-8), rarely,
and that one-ulp difference propagates through later layers. So outputs are
compared with a 2e-2 relative bound on the worst element (scaled by the
output's magnitude), and 99% of them must agree within 2e-3 of that scale.
"""
import numpy as np
import pytest

from oracle import repair as R
from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs as gsmod
    return gsmod


def _features(rng, H, W, hole_frac=0.2):
    hole = rng.random((H, W)) < hole_frac
    x = np.zeros((6, H, W))
    x[:3] = rng.random((3, H, W))
    x[3] = rng.uniform(0.2, 2.0, (H, W))
    x[:4, hole] = 0.0
    x[4] = hole
    x[5] = R.distance_to_hole(hole)
    return R.round_bf16(x), hole


def _to_device(x):
    """(6, H, W) float64 (bf16 values) -> (1, H, W, 8) bfloat16 CUDA tensor."""
    f = np.zeros((1, x.shape[1], x.shape[2], 8), np.float32)
    f[0, :, :, :6] = np.moveaxis(x, 0, -1)
    return torch.tensor(f).to(torch.bfloat16).cuda()


def _tiles(H, W, frame=0):
    ty, tx = (H + 15) // 16, (W + 15) // 16
    t = [(frame << 24) | (y << 12) | x for y in range(ty) for x in range(tx)]
    return torch.tensor(np.array(t, np.int64).astype(np.int32), device="cuda")


def _weights(seed, gate_bias=0.0):
    W, b = R.init_weights(seed)
    rng = np.random.default_rng(seed + 1)
    b = [rng.normal(0, 0.05, bb.shape) for bb in b]
    b[5][3] += gate_bias
    return W, b


def _ctx(gs, W, H):
    return gs.Context(16, W, H, max_instances=1 << 12)


def _close(gpu, ref, what):
    scale = max(float(np.abs(ref).max()), 1e-3)
    err = np.abs(gpu - ref)
    assert err.max() <= 2e-2 * scale, f"{what}: max err {err.max()} vs scale {scale}"
    assert np.quantile(err, 0.99) <= 2e-3 * scale, f"{what}: 99th pct err {np.quantile(err, 0.99)}"


@pytest.mark.parametrize("H,W", [(40, 56), (16, 16), (67, 45)])
def test_forward_matches_oracle(gs, H, W):
    rng = np.random.default_rng(H * 1000 + W)
    x, hole = _features(rng, H, W)
    Wt, b = _weights(3)
    ctx = _ctx(gs, W, H)
    ctx.repair_load(R.pack(Wt, b))
    feat = _to_device(x)
    tiles = _tiles(H, W)
    fill = torch.zeros(1, 3, H, W, device="cuda")
    _, gate = ctx.repair_infer(feat, tiles, fill=fill)
    ctx.check_ok()
    out, _ = R.forward(x, Wt, b, bf16=True)
    _close(fill[0].cpu().double().numpy(), x[:3] + out[:3], "fill")
    g_ref = R.tile_gate(out[3]).ravel()
    _close(gate.cpu().double().numpy(), g_ref, "gate")


def test_forward_is_tile_local_and_listed_only(gs):
    """Listing a subset of tiles writes exactly those tiles, with the same values."""
    rng = np.random.default_rng(9)
    H, W = 48, 64
    x, _ = _features(rng, H, W)
    Wt, b = _weights(4)
    ctx = _ctx(gs, W, H)
    ctx.repair_load(R.pack(Wt, b))
    feat = _to_device(x)
    full = torch.full((1, 3, H, W), -7.0, device="cuda")
    ctx.repair_infer(feat, _tiles(H, W), fill=full)
    part = torch.full((1, 3, H, W), -7.0, device="cuda")
    sub = torch.tensor([(1 << 12) | 2, 0], dtype=torch.int32, device="cuda")  # tiles (2, 1) and (0, 0)
    ctx.repair_infer(feat, sub, fill=part)
    ctx.check_ok()
    f, p = full.cpu().numpy(), part.cpu().numpy()
    listed = np.zeros((H, W), bool)
    listed[16:32, 32:48] = True
    listed[0:16, 0:16] = True
    assert np.array_equal(p[:, :, listed], f[:, :, listed])
    assert np.all(p[:, :, ~listed] == -7.0)


@pytest.mark.parametrize("H,W", [(32, 48), (200, 216)])
def test_gradients_match_oracle(gs, H, W):
    """Weight and bias gradients of one training step against the oracle's
    backward; 200 x 216 gives 13 x 14 = 182 tiles, more than the backward's CTAs,
    so some CTAs accumulate several tiles in tensor memory."""
    rng = np.random.default_rng(11)
    x, hole = _features(rng, H, W, 0.3)
    Wt, b = _weights(5)
    flat = R.pack(Wt, b).astype(np.float32).astype(np.float64)
    Wt, b = R.unpack(flat)
    ctx = _ctx(gs, W, H)
    ctx.repair_load(flat)
    feat = _to_device(x)
    # target far above every output (L1 sign fixed) and a perfect plain image
    # (gate label 0 on every tile), so no discrete decision sits near a boundary
    target = np.full((3, H, W), 10.0)
    tgt = torch.tensor(target[None], dtype=torch.float32, device="cuda")
    loss = ctx.repair_train_step(feat, tgt, tgt.clone(), _tiles(H, W), lr=0.0, gate_weight=0.1)
    g_gpu = ctx.repair_read(1).astype(np.float64)
    out, acts = R.forward(x, Wt, b, bf16=True)
    L, dout = R.loss(out, target, hole, np.zeros(((H + 15) // 16, (W + 15) // 16)), lam=0.1, base=x[:3])
    # the tensor-core backward rounds each layer's output gradient and its
    # weights to bfloat16 operands (FP32 accumulation); the oracle rounds at the
    # same points and sums exactly
    dW, db = R.backward(acts, Wt, dout, bf16=True)
    g_ref = R.pack(dW, db)
    assert abs(loss[0] - L) <= 1e-3 * abs(L)
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 5e-3, rel
    # every layer's weight and bias gradients, each against its own scale
    o = 0
    for l in range(6):
        ci, co = R.CHANNELS[l], R.CHANNELS[l + 1]
        for n in (co * 9 * ci, co):
            seg_g, seg_r = g_gpu[o:o + n], g_ref[o:o + n]
            assert np.abs(seg_g - seg_r).max() <= 2e-2 * np.abs(seg_r).max() + 1e-9, (l, n)
            o += n
    # lr = 0 leaves the parameters untouched
    assert np.array_equal(ctx.repair_read(0), flat.astype(np.float32))
    # the gradient sums are reduced in a fixed order: a second step gives the
    # same gradients bit for bit
    ctx.repair_train_step(feat, tgt, tgt.clone(), _tiles(H, W), lr=0.0, gate_weight=0.1)
    assert np.array_equal(ctx.repair_read(1), g_gpu.astype(np.float32))


def test_adamw_steps_reduce_the_loss(gs):
    rng = np.random.default_rng(12)
    H, W = 32, 32
    x, hole = _features(rng, H, W, 0.3)
    target = rng.random((3, H, W))
    Wt, b = _weights(6)
    ctx = _ctx(gs, W, H)
    ctx.repair_load(R.pack(Wt, b))
    feat = _to_device(x)
    tgt = torch.tensor(target[None], dtype=torch.float32, device="cuda")
    tiles = _tiles(H, W)
    scratch = ctx.repair_scratch(tiles.numel())
    losses = [ctx.repair_train_step(feat, tgt, tgt, tiles, scratch=scratch, lr=3e-3)[0] for _ in range(30)]
    assert losses[-1] < 0.6 * losses[0], losses[::5]


def test_features_match_oracle(gs, orc):
    scene, cam, dom, aff = synth.workload_small()
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22)
    ds = gs.DeviceScene(scene)
    out = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=3))
    feat = ctx.repair_features(cam)
    ctx.check_ok()
    H, W = cam.height, cam.width
    warp, _ = ctx.buffer(gs.BUF_WARP, torch.int64, None)
    strips, _ = ctx.buffer(gs.BUF_STRIPS, torch.int32, (4, 4))
    key = warp[:H * W].cpu().numpy().view(np.uint64).reshape(H, W)
    hole = key == np.uint64(0xFFFFFFFFFFFFFFFF)
    src = np.where(hole, 0, (key & np.uint64(0xFFFFFFFF)).astype(np.int64))
    rgb_dom = out["rgb_dom"].cpu().double().numpy().reshape(3, -1)
    rgb_w = np.where(hole[None], 0.0, rgb_dom[:, src.ravel()].reshape(3, H, W))
    in_strip = np.zeros((H, W), bool)
    for x0, y0, x1, y1 in strips.cpu().numpy():
        in_strip[y0:y1, x0:x1] = True
    # the method's fill of the non-strip holes (the centre-off fallback included)
    _, rgb_c = orc.classify(hole, rgb_w, in_strip, 2, center_enabled=0)
    z = (key >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)
    ref = R.round_bf16(R.features(rgb_c, z, hole))
    got = np.moveaxis(feat.float().cpu().double().numpy(), -1, 0)
    assert np.all(got[6:] == 0)
    assert np.array_equal(got[4], ref[4])
    assert hole.mean() > 0.005 and (hole & ~in_strip).sum() > 0
    # at most one bfloat16 step apart (float32 vs float64 before rounding)
    for ch in (0, 1, 2, 3, 5):
        assert np.all(np.abs(got[ch] - ref[ch]) <= 2.0 ** -7 * np.maximum(np.abs(ref[ch]), 1e-30)), ch


def _stereo(gs, ctx, ds, dom, aff, cam, mode, tau=0.5):
    roi = gs.roi_params(repair_mode=mode, gate_tau=tau)
    out = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2, roi=roi)
    ctx.check_ok()
    return {k: v.clone() for k, v in out.items()}


def test_stereo_gate_closed_and_open(gs):
    scene, cam, dom, aff = synth.workload_small()
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22)
    ds = gs.DeviceScene(scene)
    plain = _stereo(gs, ctx, ds, dom, aff, cam, 0)
    with pytest.raises(gs.GsError) as e:
        _stereo(gs, gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22), ds, dom, aff, cam, 1)
    assert e.value.status == gs.GS_ERR_NOT_LOADED
    # gate never passes: exactly the plain method
    Wt, b = _weights(7, gate_bias=-1e4)
    ctx.repair_load(R.pack(Wt, b))
    closed = _stereo(gs, ctx, ds, dom, aff, cam, 1)
    for k in ("rgb_aff", "cls_aff"):
        assert torch.equal(closed[k], plain[k]), k
    # gate always passes: the candidate tiles (re-rendered by the plain method and
    # holding a hole outside the edge strips) take max(fill, 0) at their hole
    # pixels and are not re-rendered; every other tile is the plain method's
    Wt, b = _weights(7, gate_bias=1e4)
    ctx.repair_load(R.pack(Wt, b))
    opened = _stereo(gs, ctx, ds, dom, aff, cam, 1)
    feat = ctx.repair_features(cam)
    H, W = cam.height, cam.width
    fill = torch.zeros(1, 3, H, W, device="cuda")
    ctx.repair_infer(feat[None], _tiles(H, W), fill=fill)
    pc = plain["cls_aff"]
    hole = (pc & gs.CLS_HOLE) > 0

    def per_tile(m):
        return m.reshape(H // 16, 16, W // 16, 16).any(3).any(1)

    def per_pixel(t):
        return t.repeat_interleave(16, 0).repeat_interleave(16, 1)

    cand = per_pixel(per_tile((pc & gs.CLS_RENDER) > 0) & per_tile(hole & ((pc & gs.CLS_STRIP) == 0)))
    assert cand.any() and (~cand & per_pixel(per_tile((pc & gs.CLS_RENDER) > 0))).any()
    cls = opened["cls_aff"]
    assert torch.equal((cls & gs.CLS_NET) > 0, hole & cand)
    want = torch.clamp(fill[0], min=0.0)
    assert torch.equal(opened["rgb_aff"][:, hole & cand], want[:, hole & cand])
    assert torch.equal(opened["rgb_aff"][:, ~cand], plain["rgb_aff"][:, ~cand])
    assert not torch.any((cls[cand] & gs.CLS_RENDER) > 0)


def test_gate_learns_a_rule_the_features_carry(gs):
    """Targets are built so that a tile's label is 1 exactly when under 10% of its
    pixels are holes: there the starting fill is exact, elsewhere the target
    carries zero-mean noise no fill can predict. Training must separate the two
    kinds of tile through the gate."""
    rng = np.random.default_rng(21)
    H, W = 128, 128
    frac = rng.choice([0.03, 0.3], size=(H // 16, W // 16))
    hole = rng.random((H, W)) < np.kron(frac, np.ones((16, 16)))
    x = np.zeros((6, H, W))
    x[:3] = rng.random((3, H, W))
    x[3] = rng.uniform(0.2, 2.0, (H, W))
    x[3, hole] = 0.0
    x[4] = hole
    x[5] = R.distance_to_hole(hole)
    x = R.round_bf16(x)
    pos = np.kron(frac < 0.1, np.ones((16, 16), bool))
    target = np.where(pos[None], x[:3], x[:3] + rng.uniform(-0.5, 0.5, x[:3].shape))
    plain = target + 0.05  # the plain image is never perfect
    Wt, b = R.unpack(__import__("paper_2609_30741_gb300.repair_train", fromlist=["x"]).init_weights(3))
    ctx = _ctx(gs, W, H)
    ctx.repair_load(R.pack(Wt, b))
    feat = _to_device(x)
    tgt = torch.tensor(target[None], dtype=torch.float32, device="cuda")
    pl = torch.tensor(plain[None], dtype=torch.float32, device="cuda")
    tiles = _tiles(H, W)
    scratch = ctx.repair_scratch(tiles.numel())
    for _ in range(300):
        ctx.repair_train_step(feat, tgt, pl, tiles, scratch=scratch, lr=1e-3, gate_weight=1.0, want_loss=False)
    _, gate = ctx.repair_infer(feat, tiles)
    g = gate.cpu().numpy().reshape(H // 16, W // 16)
    gp, gn = g[frac < 0.1], g[frac > 0.1]
    # rank separation (AUC) and a clear gap of the mean logits; the training
    # order of the FP32 gradient sums varies between runs, so no single tile
    # decides the outcome
    auc = (gp[:, None] > gn[None, :]).mean()
    assert auc >= 0.9 and gp.mean() > gn.mean() + 1.0, (auc, gp.mean(), gn.mean())


def test_fp8_calibration_and_forward_match_oracle(gs):
    rng = np.random.default_rng(41)
    H, W = 48, 64
    x, hole = _features(rng, H, W)
    Wt, b = _weights(8)
    flat = R.pack(Wt, b).astype(np.float32).astype(np.float64)
    Wt, b = R.unpack(flat)
    ctx = _ctx(gs, W, H)
    ctx.repair_load(flat)
    feat = _to_device(x)
    tiles = _tiles(H, W)
    with pytest.raises(gs.GsError):  # not calibrated yet
        ctx.repair_infer(feat, tiles, fp8=True)
    ctx.repair_calibrate_fp8(feat, tiles)
    sx, sw = ctx.repair_fp8_scales()
    # scales: the oracle's calibration statistic from its own BF16 network (a
    # maximum of bfloat16 activations: equal, or one bfloat16 step apart)
    amax = R.activation_maxima(x, Wt, b)
    sx_ref, sw_ref = R.fp8_scales(amax, Wt)
    used = np.zeros((6, 32), bool)
    for l in range(6):
        used[l, :R.CHANNELS[l]] = True
    np.testing.assert_allclose(sx[used], sx_ref[used], rtol=2.0 ** -7)
    out_used = np.zeros((6, 32), bool)
    for l in range(6):
        out_used[l, :R.CHANNELS[l + 1]] = True
    np.testing.assert_allclose(sw[out_used], sw_ref[out_used], rtol=2.0 ** -6)
    fill = torch.zeros(1, 3, H, W, device="cuda")
    _, gate = ctx.repair_infer(feat, tiles, fill=fill, fp8=True)
    ctx.check_ok()
    # the FP8 forward with the GPU's own scales (the network under test)
    sx64, sw64 = sx.astype(np.float64), sw.astype(np.float64)
    out = R.forward_fp8(x, Wt, b, sx64, sw64)
    _close(fill[0].cpu().double().numpy(), x[:3] + out[:3], "fp8 fill")
    _close(gate.cpu().double().numpy(), R.tile_gate(out[3]).ravel(), "fp8 gate")
    # and its error against the BF16 network, reported
    out16, _ = R.forward(x, Wt, b, bf16=True)
    rel = np.abs(out - out16).max() / np.abs(out16).max()
    print(f"fp8 vs bf16 network, max relative error {rel:.3g}")
    assert rel < 0.25


def test_stereo_fp8_mode(gs):
    scene, cam, dom, aff = synth.workload_small()
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22)
    ds = gs.DeviceScene(scene)
    plain = _stereo(gs, ctx, ds, dom, aff, cam, 0)
    Wt, b = _weights(9, gate_bias=-1e4)  # gate closed: FP8 mode equals the plain method
    ctx.repair_load(R.pack(Wt, b))
    with pytest.raises(gs.GsError) as e:
        _stereo(gs, ctx, ds, dom, aff, cam, 2)
    assert e.value.status == gs.GS_ERR_NOT_LOADED
    ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=3))
    feat = ctx.repair_features(cam)
    ctx.repair_calibrate_fp8(feat[None], _tiles(cam.height, cam.width))
    closed = _stereo(gs, ctx, ds, dom, aff, cam, 2)
    for k in ("rgb_aff", "cls_aff"):
        assert torch.equal(closed[k], plain[k]), k


def test_training_resumes_bit_for_bit(gs, tmp_path):
    """The training step is deterministic (fixed-order gradient reduction), so a
    run resumed from a checkpoint in a fresh context reproduces the
    uninterrupted run's remaining losses and final weights exactly."""
    from paper_2609_30741_gb300 import repair_train as T
    dev = torch.device("cuda", 0)
    ctx, pairs = T.build_pairs("small", 2, 2, 41, dev)
    w_full, h_full, _ = T.train(ctx, pairs, 12, 96, 2e-3, 41, log_every=1)
    ck = str(tmp_path / "ck_{step}.npz")
    T.train(ctx, pairs, 12, 96, 2e-3, 41, log_every=1, checkpoint=ck, checkpoint_every=6)
    ctx2 = gs.Context(ctx.lim.max_surfels, ctx.lim.max_width, ctx.lim.max_height, max_instances=1 << 22)
    w_res, h_res, _ = T.train(ctx2, pairs, 12, 96, 2e-3, 41, log_every=1, resume=ck.format(step=6))
    assert [h[0] for h in h_res] == list(range(6, 12))
    assert h_res == h_full[6:]
    assert np.array_equal(w_res, w_full)
