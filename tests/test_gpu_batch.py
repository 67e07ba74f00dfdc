"""Batched stereo rendering (gs_render_stereo_batch): frames of different scenes,
surfel counts and image sizes in one call, each rasterizer pass one persistent
launch over all frames. Every frame equals the single-frame call on its slot
with the same rasterizer configuration, bit for bit, in direct and graph mode;
the autotuner tries every allowed configuration and applies the fastest."""
import math

import numpy as np
import pytest

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


def _frames_spec():
    """(scene, camera, [pose pairs]) of uneven sizes; the last pair of the
    object scene is toed in (not a parallel rig)."""
    small, cam_s, dom_s, aff_s = synth.workload_small()
    obj = synth.scene_object_ground(1401, n=120_000)
    cam_o = synth.centred_camera(650, 490, 640.0)
    ball = synth.random_scene(1402, 30_000, sh_degree=3, z_range=(1.5, 4.0), scale_mu=math.log(0.03))
    cam_b = synth.centred_camera(321, 203, 260.0)
    arc = synth.arc_poses()
    toed = (synth.look_at((-0.032, 0.0, 0.0), (0.0, 0.0, 2.0)), synth.look_at((0.032, 0.0, 0.0), (0.0, 0.0, 2.0)))
    return [
        (small, cam_s, [(dom_s, aff_s), synth.eye_pair(synth.look_at((0.1, 0.0, -0.2), (0.0, 0.0, 3.0)))]),
        (obj, cam_o, [synth.eye_pair(arc[1]), toed]),
        (ball, cam_b, [synth.eye_pair(synth.look_at((0.0, 0.1, 0.0), (0.0, 0.0, 3.0))),
                       synth.eye_pair(synth.look_at((0.2, 0.0, 0.1), (0.0, 0.0, 3.0)))]),
    ]


@pytest.fixture(scope="module")
def setup(gs):
    spec = _frames_spec()
    scenes = [gs.DeviceScene(s) for s, _, _ in spec]
    # frames: every scene with its first pose pair, then every scene with its second
    items = [(k, j) for j in range(2) for k in range(len(spec))]
    ctxs, frames = [], []
    for k, j in items:
        sc, cam, poses = spec[k]
        ctx = gs.Context(sc.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
        ctxs.append(ctx)
        frames.append([scenes[k], poses[j][0], poses[j][1], cam, ctx.alloc_outputs(cam)])
    return dict(spec=spec, scenes=scenes, items=items, ctxs=ctxs, frames=frames)


KEYS = ("rgb_dom", "depth_dom", "trans_dom", "rgb_aff", "cls_aff", "roi_rects", "roi_count", "edge_widths")


def _same(kk, got, ref):
    """Outputs agree; of roi_rects only the roi_count entries written are defined."""
    if kk == "roi_rects":
        n = int(ref["roi_count"].item())
        return int(got["roi_count"].item()) == n and torch.equal(got[kk][:n], ref[kk][:n])
    return torch.equal(got[kk], ref[kk])


def _single(ctx, fr, roi=None, two_pass=False):
    ds, d, a, cam, _ = fr
    if two_pass:
        return ctx.render_two_pass(ds, d, a, cam)
    return ctx.render_stereo(ds, d, a, cam, gap_thresh=2, roi=roi)


def _assert_frames_equal(gs, setup, batch_outs, roi=None, two_pass=False, cfg=None):
    for f, (ctx, fr) in enumerate(zip(setup["ctxs"], setup["frames"])):
        if cfg is not None:
            ctx.set_raster(*cfg)
        ref = _single(ctx, fr, roi, two_pass)
        ctx.check_ok()
        keys = ("rgb_dom", "depth_dom", "trans_dom", "rgb_aff") if two_pass else KEYS
        for k in keys:
            assert _same(k, batch_outs[f], ref), (f, k)


def _clone(frames):
    return [{k: v.clone() for k, v in fr[4].items()} for fr in frames]


@pytest.mark.parametrize("cfg", [(16, 4, 128), (8, 2, 64), (32, 8, 256)])
def test_batch_equals_single_frame_calls(gs, setup, cfg):
    b = gs.Batch(setup["ctxs"])
    b.set_raster(*cfg)
    frames = [tuple(fr) for fr in setup["frames"]]
    for graphs in (False, True):
        b.set_graphs(graphs)
        for _ in range(3 if graphs else 1):  # direct, capture, replay
            b.render_stereo(frames, gap_thresh=2)
        b.check_ok()
        outs = _clone(setup["frames"])
        _assert_frames_equal(gs, setup, outs, cfg=cfg)
    b.close()


def test_graph_replay_with_new_poses(gs, setup):
    """A replayed batch graph takes each frame's new poses (patched set-up nodes)."""
    b = gs.Batch(setup["ctxs"])
    frames = [tuple(fr) for fr in setup["frames"]]
    for _ in range(2):
        b.render_stereo(frames)
    # swap every frame's poses for another pair of the same scene
    moved = []
    for (k, j), fr in zip(setup["items"], frames):
        d, a = setup["spec"][k][2][1 - j]
        moved.append((fr[0], d, a, fr[3], fr[4]))
    b.render_stereo(moved)
    b.check_ok()
    outs = _clone(setup["frames"])
    for f, (ctx, fr) in enumerate(zip(setup["ctxs"], moved)):
        ctx.set_raster(16, 4, 128)
        ref = _single(ctx, fr)
        for k in KEYS:
            assert _same(k, outs[f], ref), (f, k)
    b.close()


def test_two_pass_batch_equals_single_frame(gs, setup):
    b = gs.Batch(setup["ctxs"])
    frames = [tuple(fr) for fr in setup["frames"]]
    for _ in range(3):
        b.render_two_pass(frames)
    b.check_ok()
    outs = _clone(setup["frames"])
    _assert_frames_equal(gs, setup, outs, two_pass=True, cfg=(16, 4, 128))
    b.close()


def test_learned_repair_batch_equals_single_frame(gs, setup):
    from paper_2609_30741_gb300 import repair_train as T
    w = T.init_weights(5, gate_bias=0.0)  # gates near sigmoid(0) = 0.5: many tiles pass tau = 0.3
    rng = np.random.default_rng(6)
    w = w + rng.normal(0.0, 0.05, w.shape).astype(np.float32)  # a non-trivial fill and gate
    for ctx in setup["ctxs"]:
        ctx.repair_load(w)
    roi = gs.roi_params(repair_mode=1, gate_tau=0.3)
    b = gs.Batch(setup["ctxs"])
    frames = [tuple(fr) for fr in setup["frames"]]
    for _ in range(3):
        b.render_stereo(frames, gap_thresh=2, roi=roi)
    b.check_ok()
    outs = _clone(setup["frames"])
    _assert_frames_equal(gs, setup, outs, roi=roi, cfg=(16, 4, 128))
    b.close()


def test_batch_profiling_and_counting(gs, setup):
    b = gs.Batch(setup["ctxs"])
    frames = [tuple(fr) for fr in setup["frames"]]
    b.set_profiling(True)
    b.set_counting(True)
    for _ in range(3):
        b.render_stereo(frames)
        st = b.stage_times()
        assert len(st) == 5 and all(t >= 0.0 for t in st)
    b.check_ok()
    for ctx in setup["ctxs"]:
        ev, co = ctx.pair_counts()
        assert ev[0] >= co[0] > 0
    b.close()


def test_autotune_batch(gs, setup):
    gs.tune_cache_clear()
    b = gs.Batch(setup["ctxs"])
    frames = [tuple(fr) for fr in setup["frames"]]
    best, ms, results = b.autotune(frames, reps=3, use_cache=True)
    assert len(results) == len(gs.RASTER_CONFIGS)  # every slot allows tile 8
    assert {c for c, _ in results} == set(gs.RASTER_CONFIGS)
    assert all(t > 0 for _, t in results)
    assert ms == min(t for _, t in results) and (best, ms) in results
    assert b.raster() == best
    assert gs.tune_cache_size() == 1
    best2, ms2, results2 = b.autotune(frames, reps=3, use_cache=True)  # cached: nothing timed
    assert results2 == [] and best2 == best and ms2 == ms
    b.check_ok()
    b.close()


def test_autotune_single_frame_respects_min_tile(gs):
    gs.tune_cache_clear()
    scene, cam, dom, aff = synth.workload_small()
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22)  # min_tile 16
    ds = gs.DeviceScene(scene)
    best, ms, results = gs.autotune_stereo(ctx, ds, dom, aff, cam, reps=3, use_cache=False)
    assert {c for c, _ in results} == {c for c in gs.RASTER_CONFIGS if c[0] >= 16}
    assert ctx.raster() == best and ms > 0
    # the comparator is tuned under its own key
    best2, ms2, results2 = gs.autotune_stereo(ctx, ds, dom, aff, cam, reps=3, use_cache=True, two_pass=True)
    assert len(results2) == len(results) and ctx.raster() == best2 and ms2 > 0
    assert gs.tune_cache_size() == 2


def test_autotune_two_pass_batch(gs, setup):
    gs.tune_cache_clear()
    b = gs.Batch(setup["ctxs"])
    frames = [tuple(fr) for fr in setup["frames"]]
    best, ms, results = b.autotune(frames, reps=2, use_cache=False, two_pass=True)
    assert len(results) == len(gs.RASTER_CONFIGS) and b.raster() == best
    b.render_two_pass(frames)
    b.check_ok()
    outs = _clone(setup["frames"])
    _assert_frames_equal(gs, setup, outs, two_pass=True, cfg=best)
    b.close()


def test_batch_argument_errors(gs, setup):
    ctxs = setup["ctxs"]
    with pytest.raises(gs.GsError):
        gs.Batch([ctxs[0], ctxs[0]])  # a slot per frame
    b = gs.Batch(ctxs[:2])
    frames = [tuple(fr) for fr in setup["frames"]]
    with pytest.raises(gs.GsError):
        b.render_stereo(frames)  # more frames than slots
    with pytest.raises(gs.GsError):
        b.render_stereo(frames[1:3])  # frame 0 is the object scene: too large for slot 0
    small_ctx = gs.Context(1000, 64, 64, max_instances=1 << 16)
    b2 = gs.Batch([small_ctx])
    with pytest.raises(gs.GsError):
        b2.set_raster(8, 2, 64)  # below the slot's min_tile
    b.close()
    b2.close()


def test_autotune_skips_configs_that_overflow(gs):
    """A context whose instance capacity lies between the 32-pixel and the
    16-pixel tile counts: the 16-pixel configurations overflow, are reported
    with ms = -1, and the tuner picks a 32-pixel one."""
    gs.tune_cache_clear()
    scene, cam, dom, aff = synth.workload_small()
    ds = gs.DeviceScene(scene)
    probe = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22)
    counts = {}
    for t, p in ((16, 4), (32, 8)):
        probe.set_raster(t, p, 128)
        probe.render_mono(ds, dom, cam)
        probe.check_ok()
        counts[t] = probe.buffer(gs.BUF_INST_VALS, torch.int32)[1]
    assert counts[32] < counts[16]
    cap = (counts[32] + counts[16]) // 2
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=cap)
    best, ms, results = gs.autotune_stereo(ctx, ds, dom, aff, cam, reps=2, use_cache=False)
    assert best[0] == 32 and ms > 0
    for c, t in results:
        assert (t > 0) == (c[0] == 32), (c, t)
    ctx.check_ok()
    # nothing fits: the tuner reports the overflow and keeps the old configuration
    tiny = gs.Context(scene.n, cam.width, cam.height, max_instances=256)
    with pytest.raises(gs.GsError) as e:
        gs.autotune_stereo(tiny, ds, dom, aff, cam, reps=2, use_cache=False)
    assert e.value.status == gs.GS_ERR_CAPACITY
    assert tiny.raster() == (16, 4, 128)


def test_mono_batch_is_the_concurrent_two_eye_render(gs, setup):
    """gs_render_mono_batch with a stereo pair's two eyes as two frames renders
    both eyes in full side by side: each equals gs_render_mono of its pose, and
    the pair equals the sequential two-pass render."""
    spec = setup["spec"]
    sc, cam, poses = spec[1]  # the object scene
    ds = setup["scenes"][1]
    d, a = poses[0]
    slots = [gs.Context(sc.n, cam.width, cam.height, max_instances=1 << 24) for _ in range(2)]
    b = gs.Batch(slots)
    outs = [(torch.empty(3, cam.height, cam.width, device="cuda"), torch.empty(cam.height, cam.width, device="cuda"),
             torch.empty(cam.height, cam.width, device="cuda")) for _ in range(2)]
    for _ in range(3):  # direct, capture, replay
        b.render_mono([(ds, d, cam, outs[0], None), (ds, a, cam, outs[1], None)])
    b.check_ok()
    got = [[t.clone() for t in o] for o in outs]
    ref_ctx = gs.Context(sc.n, cam.width, cam.height, max_instances=1 << 24)
    for pose, g in zip((d, a), got):
        r = ref_ctx.render_mono(ds, pose, cam)
        for x, y in zip(g, r):
            assert torch.equal(x, y)
    tp = ref_ctx.render_two_pass(ds, d, a, cam)
    assert torch.equal(got[0][0], tp["rgb_dom"]) and torch.equal(got[0][1], tp["depth_dom"])
    assert torch.equal(got[1][0], tp["rgb_aff"])
    b.close()
