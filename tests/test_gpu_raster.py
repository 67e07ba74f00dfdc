"""The persistent rasterizer's configurations - tile edge 8, 16 or 32 pixels,
pixels per thread (block shape) and surfel records per shared-memory stage -
produce the same images bit for bit. A tile's list holds every surfel that can
reach one of its pixel centres, in depth order, so the tiling never changes
which surfels a pixel blends or their order, and a pixel's arithmetic depends
on its position only (the homogeneous plane point is evaluated per pixel). The
contributed-pair count, a sum over pixels, is equal too; the evaluated-pair
count grows with the tile edge."""
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


def _case(name):
    if name == "small":
        scene, cam, dom, aff = synth.workload_small()
        return scene, cam, dom, aff
    if name == "object_ragged":  # ragged tiles on both axes at every tile edge
        scene = synth.scene_object_ground(1301, n=80_000)
        cam = synth.centred_camera(650, 490, 640.0)
        dom, aff = synth.eye_pair(synth.arc_poses()[2])
        return scene, cam, dom, aff
    # toed-in eyes: not a parallel rig, each eye sorts by its own depth keys
    scene = synth.scene_object_ground(1302, n=50_000)
    cam = synth.centred_camera(480, 360, 480.0)
    dom = synth.look_at((-0.032, 0.0, 0.0), (0.0, 0.0, 2.0))
    aff = synth.look_at((0.032, 0.0, 0.0), (0.0, 0.0, 2.0))
    return scene, cam, dom, aff


def _mismatch(ref, got, k):
    """Where two stereo outputs differ: pixel count, class bits and 16-pixel tiles."""
    d = ref[k] != got[k]
    if k not in ("rgb_aff", "cls_aff") or "cls_aff" not in ref:
        return f"{k}: {ref[k].flatten()[:8].tolist()} vs {got[k].flatten()[:8].tolist()}"
    d = d.any(0) if d.dim() == 3 else d
    ys, xs = (v.cpu().numpy() for v in torch.nonzero(d, as_tuple=True))
    ca, cb = ref["cls_aff"][ys, xs].cpu().numpy(), got["cls_aff"][ys, xs].cpu().numpy()
    tiles = sorted(set(zip((ys // 16).tolist(), (xs // 16).tolist())))
    return (f"{k}: {len(ys)} pixels in {len(tiles)} tiles {tiles[:8]}, classes {np.unique(ca).tolist()} vs "
            f"{np.unique(cb).tolist()}, cls_aff equal: {torch.equal(ref['cls_aff'], got['cls_aff'])}")


def _run(ctx, ds, dom, aff, cam):
    ctx.set_counting(True)
    o = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2)
    ev, co = ctx.pair_counts()
    t = ctx.render_two_pass(ds, dom, aff, cam)
    m = ctx.render_mono(ds, aff, cam, bg=(0.1, 0.2, 0.3))
    ctx.check_ok()
    ctx.set_counting(False)
    imgs = {k: v.clone() for k, v in o.items() if k in ("rgb_dom", "depth_dom", "trans_dom", "rgb_aff", "cls_aff",
                                                         "edge_widths", "roi_count")}
    imgs.update(tp_dom=t["rgb_dom"].clone(), tp_aff=t["rgb_aff"].clone(), mono=m[0].clone(), mono_d=m[1].clone(),
                mono_t=m[2].clone())
    return imgs, ev, co


@pytest.mark.parametrize("case", ["small", "object_ragged", "toed_in"])
def test_every_raster_config_is_bit_identical(gs, case):
    scene, cam, dom, aff = _case(case)
    ds = gs.DeviceScene(scene)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    assert ctx.raster() == (16, 4, 128)
    ref, ev_ref, co_ref = _run(ctx, ds, dom, aff, cam)
    assert co_ref[0] > 0 and co_ref[1] > 0
    for cfg in gs.RASTER_CONFIGS:
        ctx.set_raster(*cfg)
        assert ctx.raster() == cfg
        got, ev, co = _run(ctx, ds, dom, aff, cam)
        for k in ref:
            assert torch.equal(ref[k], got[k]), (cfg, _mismatch(ref, got, k))
        assert co == co_ref, (cfg, co, co_ref)
        assert ev[0] >= co[0] and ev[1] >= co[1]


def test_tile_edge_orders_the_evaluated_pairs(gs):
    scene, cam, dom, aff = _case("object_ragged")
    ds = gs.DeviceScene(scene)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    ev = {}
    for t, p in ((8, 2), (16, 4), (32, 8)):
        ctx.set_raster(t, p, 128)
        _, e, _ = _run(ctx, ds, dom, aff, cam)
        ev[t] = e[0]
    assert ev[8] < ev[16] < ev[32], ev


def test_invalid_raster_configs_are_rejected(gs):
    ctx = gs.Context(1000, 128, 96, max_instances=1 << 16)  # min_tile 16
    for bad in ((8, 2, 128), (16, 3, 128), (16, 4, 100), (32, 1, 64), (12, 4, 128), (16, 4, 512)):
        with pytest.raises(gs.GsError):
            ctx.set_raster(*bad)
    ctx.set_raster(32, 4, 64)
    assert ctx.raster() == (32, 4, 64)
    with pytest.raises(gs.GsError):  # a context sized for 32-pixel tiles cannot run smaller ones
        gs.Context(1000, 128, 96, max_instances=1 << 16, min_tile=32).set_raster(16, 4, 128)
    with pytest.raises(gs.GsError):  # 8-pixel tiles: at most 512 tile columns
        gs.Context(1000, 4104, 96, max_instances=1 << 16, min_tile=8)


def test_masked_pass_at_tile_32_writes_only_roi_tiles(gs):
    """With 32-pixel tiles the ROI pass renders whole 32-pixel tiles but writes
    only the pixels of the ROI's 16-pixel tiles; the re-rendered class bit marks
    exactly the 16-pixel ROI tiles."""
    scene, cam, dom, aff = _case("object_ragged")
    ds = gs.DeviceScene(scene)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    ctx.set_raster(32, 8, 128)
    o = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2)
    ctx.check_ok()
    mask, _ = ctx.buffer(gs.BUF_TILE_MASK, torch.uint8)
    tx, ty = math.ceil(cam.width / 16), math.ceil(cam.height / 16)
    m = mask[:tx * ty].view(ty, tx).bool()
    rendered = (o["cls_aff"] & gs.CLS_RENDER) > 0
    expect = m.repeat_interleave(16, 0).repeat_interleave(16, 1)[:cam.height, :cam.width]
    assert 0 < int(m.sum()) < tx * ty
    assert torch.equal(rendered, expect)


def test_programmatic_launch_changes_nothing(gs):
    """Programmatic dependent launch only lets a kernel start its set-up early:
    every kernel waits for its predecessor before touching memory, so frames
    are identical with it on and off (direct launches and graph replays)."""
    scene, cam, dom, aff = _case("object_ragged")
    ds = gs.DeviceScene(scene)
    res = {}
    for on in (False, True):
        gs.set_programmatic_launch(on)
        assert gs.programmatic_launch() == on
        ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24)
        ctx.set_raster(32, 4, 64)
        for _ in range(3):  # direct, capture, replay
            got, _, _ = _run(ctx, ds, dom, aff, cam)
        res[on] = got
    gs.set_programmatic_launch(True)
    for k in res[True]:
        assert torch.equal(res[True][k], res[False][k]), k


@pytest.mark.parametrize("case", ["small", "object_ragged", "toed_in"])
def test_roi_raster_config_is_bit_identical(gs, case):
    """The ROI re-render in its own configuration (another tile edge than the
    dominant eye's, 16-pixel tiles reading a 32-pixel binning's lists, also in
    depth_mode 2 where the strips render on a second stream, and with the learned
    repair running beside the ROI binning) gives the same stereo frame bit for
    bit."""
    scene, cam, dom, aff = _case(case)
    ds = gs.DeviceScene(scene)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    from paper_2609_30741_gb300 import repair_train as T
    w = T.init_weights(5, gate_bias=0.0)
    w += np.random.default_rng(6).normal(0.0, 0.03, w.shape).astype(np.float32)
    ctx.repair_load(w)
    for mode, repair in ((0, 0), (2, 0), (0, 1)):
        roi = gs.roi_params(depth_mode=mode, repair_mode=repair, gate_tau=0.4)
        for dom_cfg in ((32, 2, 64), (16, 4, 128)):
            ctx.set_raster(*dom_cfg)
            ctx.set_raster_roi(None)
            for _ in range(2):  # depth_mode 2: the second call reuses the first one's range
                ref = {k: v.clone() for k, v in ctx.render_stereo(ds, dom, aff, cam, roi=roi).items()}
            ctx.check_ok()
            for roi_cfg in ((16, 2, 64), (8, 2, 128), (32, 4, 256)):
                ctx.set_raster_roi(roi_cfg)
                assert ctx.raster_roi() == (roi_cfg, True)
                for _ in range(2):
                    got = ctx.render_stereo(ds, dom, aff, cam, roi=roi)
                ctx.check_ok()
                for k in ("rgb_dom", "rgb_aff", "cls_aff", "roi_count", "edge_widths"):
                    assert torch.equal(ref[k], got[k]), (mode, repair, dom_cfg, roi_cfg, _mismatch(ref, got, k))
            if repair:  # the gate passed somewhere, so the skip path was exercised
                assert bool(((ref["cls_aff"] & gs.CLS_NET) > 0).any())
    ctx.set_raster_roi(None)
    assert ctx.raster_roi() == (ctx.raster(), False)


@pytest.mark.parametrize("repair", [0, 1])
def test_frames_are_the_same_under_concurrent_load(gs, repair):
    """Kernels of another stream sharing the SMs change every warp's timing, not
    the frame: the toed-in stereo frame (its affiliated eye sorted by its own
    depth keys, the learned repair beside the ROI binning when asked) rendered
    while a second stream runs elementwise work equals the frame rendered alone,
    bit for bit, every time."""
    scene, cam, dom, aff = _case("toed_in")
    ds = gs.DeviceScene(scene)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 24, min_tile=8)
    if repair:
        from paper_2609_30741_gb300 import repair_train as T
        w = T.init_weights(5, gate_bias=0.0)
        w += np.random.default_rng(6).normal(0.0, 0.03, w.shape).astype(np.float32)
        ctx.repair_load(w)
    roi = gs.roi_params(repair_mode=repair, gate_tau=0.4)
    ctx.set_raster(32, 2, 64)
    out = ctx.alloc_outputs(cam)
    for _ in range(3):
        ctx.render_stereo(ds, dom, aff, cam, roi=roi, out=out)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in out.items()}
    side = torch.cuda.Stream()
    load = torch.randn(2048, 2048, device="cuda")
    for it in range(30):
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(4):
                load = torch.sin(load) * 1.0001
        ctx.render_stereo(ds, dom, aff, cam, roi=roi, out=out)
        torch.cuda.current_stream().wait_stream(side)
        ctx.check_ok()
        for k in ("rgb_dom", "rgb_aff", "cls_aff", "roi_count"):
            assert torch.equal(ref[k], out[k]), (it, _mismatch(ref, out, k))
