"""The headset workload at full size: 3M surfels of the unbounded distribution,
2448x2448 per eye (f = 1800), frames of the 120-frame head trajectory (60 deg/s
at 90 Hz). Per frame, against the FP64 oracle on a 256x256 crop centred on a
seeded ROI pixel and against the GPU's full render of the affiliated eye:

- the two-pass comparator's crop equals the oracle within the parity tolerance;
- the plain method's re-rendered (ROI) pixels equal the oracle too;
- the FP8 (e4m3, per-channel scales) repair network stays within a small
  distance of the BF16 one, pixel by pixel and in PSNR against the oracle.

The network here is an untrained one with a small random last layer and an open
gate, so that it fills many tiles (its quality is the training's business; this
is about the precision ladder at this size)."""
import math

import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RGB_TOL = 2e-4
# Pixels with a blend decision within MARGIN (relative) of its threshold, or with
# near-equal depth keys among their contributors, are excluded from the
# tolerance. The smaller parity workloads use 1e-5 and bound the excluded share
# at 0.1 %. Here a pixel evaluates about 400 surfels, and float32 rounding of
# the running transmittance accumulates to about 400 * 2^-24 = 2.4e-5 relative,
# so decisions within 1e-4 may flip; and the 1.8M surfels of the 1 m ball give
# many near-equal depth keys. The excluded share is printed and bounded loosely;
# at least 10,000 pixels of every crop are held to the tolerance.
MARGIN = 1e-4
MAX_MARGINAL = 0.5
MIN_CHECKED = 10_000


@pytest.fixture(scope="module")
def hmd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs, repair_train as T
    scene = synth.scene_unbounded(1500, 3_000_000)
    cam = synth.centred_camera(2448, 2448, 1800.0)
    traj = synth.yaw_trajectory(120, 60.0, 90.0, 3.0)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 28)
    ds = gs.DeviceScene(scene)
    w = T.init_weights(11, gate_bias=1.0)
    rng = np.random.default_rng(12)
    w[-(32 * 9 * 4 + 4):-4] += rng.normal(0.0, 0.02, 32 * 9 * 4).astype(np.float32)  # a non-zero last layer
    ctx.repair_load(w)
    # FP8 scales from the BF16 network on the first frame's features
    d, a = synth.eye_pair(traj[0])
    ctx.render_stereo(ds, d, a, cam, roi=gs.roi_params(repair_mode=3))
    feat = ctx.repair_features(cam)
    H, W = cam.height, cam.width
    tiles = torch.tensor([(y << 12) | x for y in range(0, (H + 15) // 16, 3) for x in range((W + 15) // 16)],
                         dtype=torch.int32, device=feat.device)
    ctx.repair_calibrate_fp8(feat[None], tiles)
    return dict(gs=gs, scene=scene, cam=cam, traj=traj, ctx=ctx, ds=ds)


def _crop(t, x0, y0, n=256):
    return t[..., y0:y0 + n, x0:x0 + n].detach().double().cpu().numpy()


def _psnr(a, b):
    return 10 * math.log10(1.0 / max(float(np.mean((a - b) ** 2)), 1e-20))


@pytest.mark.parametrize("frame", [0, 119])
def test_hmd_frame_against_oracle_crop(hmd, orc, frame):
    gs, ctx, ds, cam = hmd["gs"], hmd["ctx"], hmd["ds"], hmd["cam"]
    d, a = synth.eye_pair(hmd["traj"][frame])
    full = {k: v.clone() for k, v in ctx.render_two_pass(ds, d, a, cam).items()}
    outs = {}
    for name, mode in (("plain", 0), ("bf16", 1), ("fp8", 2)):
        o = ctx.render_stereo(ds, d, a, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=mode, gate_tau=0.5))
        outs[name] = {k: v.clone() for k, v in o.items()}
    ctx.check_ok()
    # a 256x256 crop centred on a seeded re-rendered pixel of the plain method
    ren = ((outs["plain"]["cls_aff"] & gs.CLS_RENDER) > 0).nonzero()
    assert ren.shape[0] > 0
    pick = ren[np.random.default_rng(100 + frame).integers(ren.shape[0])].tolist()
    y0 = int(np.clip(pick[0] - 128, 0, cam.height - 256))
    x0 = int(np.clip(pick[1] - 128, 0, cam.width - 256))
    o_rgb, o_dep, o_tr, mrg, _ = orc.render(hmd["scene"], a, cam, window=(x0, y0, 256, 256))
    ok = mrg >= MARGIN
    print({"frame": frame, "excluded_share": float(1.0 - ok.mean())})
    assert 1.0 - ok.mean() <= MAX_MARGINAL and int(ok.sum()) >= MIN_CHECKED
    # the comparator's crop is the oracle's full render
    e_full = np.abs(_crop(full["rgb_aff"], x0, y0) - o_rgb).max(0)[ok].max()
    assert e_full <= RGB_TOL, e_full
    # the plain method's re-rendered pixels are exact
    rend = (_crop(outs["plain"]["cls_aff"], x0, y0).astype(np.int64) & gs.CLS_RENDER) > 0
    e_roi = np.abs(_crop(outs["plain"]["rgb_aff"], x0, y0) - o_rgb).max(0)[rend & ok].max(initial=0.0)
    assert rend.any() and e_roi <= RGB_TOL, e_roi
    # precision ladder: FP8 within reach of BF16
    p = {k: _psnr(_crop(v["rgb_aff"], x0, y0), o_rgb) for k, v in outs.items()}
    p_full = {k: _psnr(v["rgb_aff"].double().cpu().numpy(), full["rgb_aff"].double().cpu().numpy())
              for k, v in outs.items()}
    net = (outs["bf16"]["cls_aff"] & gs.CLS_NET) > 0
    diff = (outs["fp8"]["rgb_aff"] - outs["bf16"]["rgb_aff"]).abs()[:, net]
    print({"frame": frame, "crop": (x0, y0), "psnr_vs_oracle_crop": p, "psnr_vs_full_frame": p_full,
           "net_px": int(net.sum()), "fp8_vs_bf16_max": float(diff.max()) if diff.numel() else 0.0})
    assert int(net.sum()) > 0
    # e4m3 keeps 3 mantissa bits: about 6 % relative error per rounding, so the
    # fill differs by a few percent of the network's correction, not more
    assert float(diff.mean()) <= 0.02 and float(diff.max()) <= 0.2
    assert p["fp8"] >= p["bf16"] - 0.5 and p_full["fp8"] >= p_full["bf16"] - 0.5
