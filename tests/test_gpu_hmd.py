"""The headset workload at full size: 3M surfels of the unbounded distribution,
2448x2448 per eye (f = 1800), frames of the 120-frame head trajectory (60 deg/s
at 90 Hz). Per frame, against the FP64 oracle on a 256x256 crop centred on a
seeded ROI pixel and against the GPU's full render of the affiliated eye:

- the two-pass comparator's crop equals the oracle within the parity tolerance;
- the plain method's re-rendered (ROI) pixels equal the oracle too;
- for the plain method and the trained network in BF16 and in FP8 (e4m3,
  per-channel scales), the per-frame max-abs error and PSNR of the crop against
  the oracle and of the whole frame against the full render are reported, on a
  seeded sample of 16 of the 120 frames;
- the FP8 network stays within a small distance of the BF16 one, pixel by pixel
  and in PSNR against the oracle (also with an untrained network whose open gate
  fills many tiles).
"""
import math

import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RGB_TOL = 2e-4
# Excluded from the tolerance (the scope of the float32 reading of the
# tolerance): pixels with a blend decision within MARGIN (relative) of its
# threshold, near-equal depth keys among their contributors, and pixels whose
# float32 evaluation cannot meet the tolerance by construction (the oracle's
# first-order estimate, or_render's fp32_bound, above the tolerance). At this
# size the float32 conditioning of the ray-plane solve decides: a pixel
# evaluates about 400 surfels, 10-30 m away and a few cm large, many of them
# seen nearly edge-on from 3 m with f = 1800, where float32 rho3 errs by up to
# about 1 % (one surfel with the ray 0.3 degrees off its plane and weight 0.28
# moved a pixel of frame 17 by 2.8e-4; a skip decision 4.4e-4 from its
# threshold flipped on frame 14). With the bound requested the oracle's margins
# subtract each surfel's rho3 error bound and fp32_bound includes the largest
# single-surfel effect of it, so both pixels are excluded. The excluded shares
# of every crop are printed and bounded by MAX_MARGINAL.
MARGIN = 1e-4
FP32_BOUND_MAX = RGB_TOL
MAX_MARGINAL = 0.10
N_FRAMES = 16


@pytest.fixture(scope="module")
def hmd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs, repair_train as T
    dev = torch.device("cuda", 0)
    # the network the bench uses on this distribution: the packaged one, trained
    # by the library's kernels on 2,000 pairs of unbounded scenes (seeds
    # 7000-7049); FP8 scales calibrated on 8 frames of another seed
    w_trained = np.load(T.UNBOUNDED_WEIGHTS)
    tctx, pairs = T.build_pairs("unbounded", 1, 8, 7100, dev)
    tiles = pairs.tile_tensor()
    calib = (pairs.feat[:8].clone(), tiles[tiles < (8 << 24)][::4].contiguous())
    del tctx, pairs
    torch.cuda.empty_cache()
    scene = synth.scene_unbounded(1500, 3_000_000)
    cam = synth.centred_camera(2448, 2448, 1800.0)
    traj = synth.yaw_trajectory(120, 60.0, 90.0, 3.0)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 28)
    ds = gs.DeviceScene(scene)
    return dict(gs=gs, T=T, scene=scene, cam=cam, traj=traj, ctx=ctx, ds=ds, w_trained=w_trained, calib=calib)


def _crop(t, x0, y0, n=256):
    return t[..., y0:y0 + n, x0:x0 + n].detach().double().cpu().numpy()


def _psnr(a, b):
    return 10 * math.log10(1.0 / max(float(np.mean((a - b) ** 2)), 1e-20))


def _render_arms(hmd, frame):
    gs, ctx, ds, cam = hmd["gs"], hmd["ctx"], hmd["ds"], hmd["cam"]
    d, a = synth.eye_pair(hmd["traj"][frame])
    full = {k: v.clone() for k, v in ctx.render_two_pass(ds, d, a, cam).items()}
    outs = {}
    for name, mode in (("plain", 0), ("bf16", 1), ("fp8", 2)):
        o = ctx.render_stereo(ds, d, a, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=mode, gate_tau=0.5))
        outs[name] = {k: v.clone() for k, v in o.items()}
    ctx.check_ok()
    return a, full, outs


def _roi_crop(gs, cam, outs, frame):
    """A 256x256 crop centred on a seeded re-rendered pixel of the plain method."""
    ren = ((outs["plain"]["cls_aff"] & gs.CLS_RENDER) > 0).nonzero()
    assert ren.shape[0] > 0
    pick = ren[np.random.default_rng(100 + frame).integers(ren.shape[0])].tolist()
    y0 = int(np.clip(pick[0] - 128, 0, cam.height - 256))
    x0 = int(np.clip(pick[1] - 128, 0, cam.width - 256))
    return x0, y0


def _maxabs(a, b):
    return float(np.abs(a - b).max())


def test_hmd_frames_against_oracle_crops(hmd, orc):
    """A seeded sample of 16 of the 120 frames (always the first and the last):
    per frame and per arm (plain, trained BF16, trained FP8) the max-abs error
    and PSNR of a 256x256 crop against the FP64 oracle's full render of the
    affiliated eye, and the PSNR of the whole frame against the GPU's full render.
    The comparator's crop and the plain method's re-rendered pixels must equal
    the oracle within the parity tolerance on every frame."""
    gs, ctx, cam = hmd["gs"], hmd["ctx"], hmd["cam"]
    ctx.repair_load(hmd["w_trained"])
    ctx.repair_calibrate_fp8(*hmd["calib"])
    rng = np.random.default_rng(2448)
    frames = sorted({0, 119} | set(rng.choice(np.arange(1, 119), N_FRAMES - 2, replace=False).tolist()))
    assert len(frames) == N_FRAMES
    rows = []
    for frame in frames:
        a, full, outs = _render_arms(hmd, frame)
        x0, y0 = _roi_crop(gs, cam, outs, frame)
        o_rgb, _, _, mrg, _, bound = orc.render(hmd["scene"], a, cam, window=(x0, y0, 256, 256), fp32_bound=True)
        ok = (mrg >= MARGIN) & (bound <= FP32_BOUND_MAX)
        excluded = float(1.0 - ok.mean())
        e_map = np.abs(_crop(full["rgb_aff"], x0, y0) - o_rgb).max(0)
        e_full = e_map[ok].max()
        worst = np.unravel_index(np.argmax(np.where(ok, e_map, -1.0)), e_map.shape)
        rend = (_crop(outs["plain"]["cls_aff"], x0, y0).astype(np.int64) & gs.CLS_RENDER) > 0
        e_roi = np.abs(_crop(outs["plain"]["rgb_aff"], x0, y0) - o_rgb).max(0)[rend & ok].max(initial=0.0)
        row = {"frame": frame, "crop": (x0, y0), "excluded_share": round(excluded, 4),
               "comparator_max_abs": float(e_full), "plain_roi_max_abs": float(e_roi),
               "worst": {"yx": [int(worst[0]), int(worst[1])], "margin": float(mrg[worst]),
                         "fp32_bound": float(bound[worst])},
               "share_marginal": round(float((mrg < MARGIN).mean()), 4),
               "share_fp32_bound": round(float((bound > FP32_BOUND_MAX).mean()), 4),
               "fp32_bound_max": float(bound.max())}
        f_ref = full["rgb_aff"].double().cpu().numpy()
        for k, v in outs.items():
            c = _crop(v["rgb_aff"], x0, y0)
            row[k] = {"crop_max_abs": round(_maxabs(c, o_rgb), 5), "crop_psnr_db": round(_psnr(c, o_rgb), 3),
                      "frame_psnr_vs_full_db": round(_psnr(v["rgb_aff"].double().cpu().numpy(), f_ref), 3),
                      "net_px": int(((v["cls_aff"] & gs.CLS_NET) > 0).sum())}
        print(row)
        rows.append(row)
        assert excluded <= MAX_MARGINAL and int(ok.sum()) >= 10_000, row
        assert e_full <= RGB_TOL, row
        assert rend.any() and e_roi <= RGB_TOL, row
        assert row["fp8"]["crop_psnr_db"] >= row["bf16"]["crop_psnr_db"] - 0.5, row
    print({"frames": frames,
           "max_excluded_share": max(r["excluded_share"] for r in rows),
           **{k: {"crop_max_abs_max": max(r[k]["crop_max_abs"] for r in rows),
                  "crop_psnr_mean_db": float(np.mean([r[k]["crop_psnr_db"] for r in rows])),
                  "frame_psnr_mean_db": float(np.mean([r[k]["frame_psnr_vs_full_db"] for r in rows]))}
              for k in ("plain", "bf16", "fp8")}})


@pytest.mark.parametrize("frame", [0, 119])
def test_hmd_fp8_precision_ladder_open_gate(hmd, orc, frame):
    """An untrained network with a small random last layer and an open gate, so
    that it fills many tiles: FP8 within reach of BF16 pixel by pixel and in
    PSNR (this is about the precision ladder at this size, not quality)."""
    gs, ctx, ds, cam = hmd["gs"], hmd["ctx"], hmd["ds"], hmd["cam"]
    w = hmd["T"].init_weights(11, gate_bias=1.0)
    rng = np.random.default_rng(12)
    w[-(32 * 9 * 4 + 4):-4] += rng.normal(0.0, 0.02, 32 * 9 * 4).astype(np.float32)  # a non-zero last layer
    ctx.repair_load(w)
    # FP8 scales from the BF16 network on the first frame's features
    d, a = synth.eye_pair(hmd["traj"][0])
    ctx.render_stereo(ds, d, a, cam, roi=gs.roi_params(repair_mode=3))
    feat = ctx.repair_features(cam)
    H, W = cam.height, cam.width
    tiles = torch.tensor([(y << 12) | x for y in range(0, (H + 15) // 16, 3) for x in range((W + 15) // 16)],
                         dtype=torch.int32, device=feat.device)
    ctx.repair_calibrate_fp8(feat[None], tiles)
    a, full, outs = _render_arms(hmd, frame)
    x0, y0 = _roi_crop(gs, cam, outs, frame)
    o_rgb, _, _, mrg, _ = orc.render(hmd["scene"], a, cam, window=(x0, y0, 256, 256))
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
