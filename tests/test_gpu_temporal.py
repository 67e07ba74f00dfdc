"""Temporal reuse of the depth range (depth_mode 2): a stereo call takes the
range the previous call measured, so its edge strips (Eq. 6-8) are known before
the dominant eye is rendered and the affiliated eye's strip tiles are rendered on
a second stream meanwhile. Every frame equals the plain pipeline with a fixed
range (depth_mode 1, itself held to the oracle) set to the previous frame's
measured range, bit for bit, in direct and graph mode; a context's first call
measures its own range."""
import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("rgb_dom", "depth_dom", "trans_dom", "rgb_aff", "cls_aff", "roi_rects", "roi_count", "edge_widths")


def _same(kk, got, ref):
    """Outputs agree; of roi_rects only the roi_count entries written are defined."""
    if kk == "roi_rects":
        n = int(ref["roi_count"].item())
        return int(got["roi_count"].item()) == n and torch.equal(got[kk][:n], ref[kk][:n])
    return torch.equal(got[kk], ref[kk])


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs as gsmod
    return gsmod


def _trajectory(kind):
    if kind == "object":
        scene = synth.scene_object_ground(1601, n=150_000)
        cam = synth.centred_camera(800, 600, 800.0)
        return scene, cam, [synth.eye_pair(p) for p in synth.arc_poses(6)]
    scene = synth.scene_object_ground(1602, n=60_000)
    cam = synth.centred_camera(480, 360, 480.0)
    toed = []
    for k in range(5):  # toed-in pairs: not a parallel rig
        c = np.array([0.05 * k, 0.0, 0.0])
        toed.append((synth.look_at(c + (-0.032, 0, 0), (0.0, 0.0, 2.0)), synth.look_at(c + (0.032, 0, 0), (0.0, 0.0, 2.0))))
    return scene, cam, toed


def _measured_range(gs, ctx, ds, pair, cam, roi0):
    out = ctx.render_stereo(ds, pair[0], pair[1], cam, gap_thresh=2, roi=roi0)
    rng, _ = ctx.buffer(gs.BUF_DEPTH_RANGE, torch.float32)
    return [float(v) for v in rng[:2].cpu()], out


@pytest.mark.parametrize("kind,cfg,repair", [("object", (16, 4, 128), 0), ("object", (32, 4, 64), 0),
                                             ("toed_in", (16, 4, 128), 0), ("object", (8, 2, 64), 0),
                                             ("object", (32, 4, 64), 1)])
def test_reuse_equals_fixed_range_of_previous_frame(gs, kind, cfg, repair):
    from paper_2609_30741_gb300 import repair_train as T
    scene, cam, pairs = _trajectory(kind)
    ds = gs.DeviceScene(scene)
    a = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    b = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    a.set_raster(*cfg)
    b.set_raster(*cfg)
    if repair:
        w = T.init_weights(21, gate_bias=0.0)
        w += np.random.default_rng(22).normal(0.0, 0.03, w.shape).astype(np.float32)
        a.repair_load(w)
        b.repair_load(w)
    reuse = gs.roi_params(depth_mode=2, repair_mode=repair, gate_tau=0.4)
    prev = None
    for k, (d, f) in enumerate(pairs + pairs[::-1]):  # forth and back: direct, capture and replays
        got = {kk: v.clone() for kk, v in a.render_stereo(ds, d, f, cam, gap_thresh=2, roi=reuse).items()}
        a.check_ok()
        if prev is None:  # the first call measures its own range: mode 0
            ref = b.render_stereo(ds, d, f, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=repair, gate_tau=0.4))
        else:
            ref = b.render_stereo(ds, d, f, cam, gap_thresh=2,
                                  roi=gs.roi_params(depth_mode=1, d_min=prev[0], d_max=prev[1], repair_mode=repair,
                                                    gate_tau=0.4))
        b.check_ok()
        for kk in KEYS:
            assert _same(kk, got, ref), (k, kk)
        # the range this frame measured, for the next one
        prev, _ = _measured_range(gs, b, ds, (d, f), cam, gs.roi_params(repair_mode=repair, gate_tau=0.4))


def test_reuse_in_batches(gs):
    """A batch with depth_mode 2 equals its frames' single-context calls."""
    scene, cam, pairs = _trajectory("object")
    ds = gs.DeviceScene(scene)
    slots = [gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24) for _ in range(2)]
    refs = [gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24) for _ in range(2)]
    bt = gs.Batch(slots)
    roi = gs.roi_params(depth_mode=2)
    for k in range(4):
        frames = [(ds, *pairs[(k + j) % len(pairs)], cam, slots[j].alloc_outputs(cam)) for j in range(2)]
        bt.render_stereo(frames, gap_thresh=2, roi=roi)
        bt.check_ok()
        for j in range(2):
            r = refs[j].render_stereo(ds, *pairs[(k + j) % len(pairs)], cam, gap_thresh=2, roi=roi)
            for kk in KEYS:
                assert _same(kk, frames[j][4], r), (k, j, kk)
    bt.close()
