"""The 3DGS backbone (3D Gaussian ellipsoids, EWA splatting) on the CUDA path
against the FP64 oracle, through the C ABI.

Sec. 3.2: the pipeline accepts any Gaussian splatting variant that outputs
per-pixel depth. The ellipsoid scenes are the synthetic surfel scenes with a
third axis (synth.to_ellipsoids); renders are compared with the oracle's
ellipsoid path within the surfel tolerances, on pixels away from a decision
threshold. The stereo method on an ellipsoid scene is checked like the surfel
one: ROI tiles equal the full affiliated render bit for bit (same kernels), and
the whole method agrees with the oracle's own pipeline.
"""
import math

import numpy as np
import pytest

from paper_2609_30741_gb300 import synth
from test_gpu_parity import RGB_TOL, _np, compare_render, make_ctx

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


def _case(which):
    if which == "small":
        scene, cam, dom, aff = synth.workload_small()
        return synth.to_ellipsoids(scene, 0.1), cam, dom, aff
    if which == "small_ragged":
        scene, cam, dom, aff = synth.workload_small()
        return synth.to_ellipsoids(scene, 1.0), synth.centred_camera(250, 171, 300.0), dom, aff
    scene = synth.random_scene(23, 3000, sh_degree=3, z_range=(1.0, 5.0), scale_mu=math.log(0.04))
    cam = synth.centred_camera(200, 136, 180.0)
    dom = synth.look_at((0.2, -0.1, -0.3), (0.0, 0.0, 3.0))
    return synth.to_ellipsoids(scene, 0.5), cam, dom, None


@pytest.mark.parametrize("which", ["small", "small_ragged", "random_sh3", "small@8,1,32", "small_ragged@32,8,256",
                                   "random_sh3@32,4,128"])
def test_ellipsoid_render_matches_oracle(gs, orc, which):
    which, _, cfg = which.partition("@")
    scene, cam, dom, _ = _case(which)
    ctx = make_ctx(gs, scene, cam, min_tile=8)
    if cfg:
        ctx.set_raster(*(int(v) for v in cfg.split(",")))
    rgb, dep, tr = ctx.render_mono(gs.DeviceScene(scene), dom, cam, bg=(0.1, 0.2, 0.3))
    ctx.check_ok()
    o_rgb, o_dep, o_tr, mrg, _ = orc.render(scene, dom, cam, bg=(0.1, 0.2, 0.3))
    assert (1.0 - o_tr).mean() > 0.05, "the case covers too little of the image"
    compare_render(_np(rgb), _np(dep), _np(tr), o_rgb, o_dep, o_tr, mrg, which)


def test_ellipsoid_render_identical_across_raster_configs(gs):
    scene, cam, dom, _ = _case("small_ragged")
    ctx = make_ctx(gs, scene, cam, min_tile=8)
    ds = gs.DeviceScene(scene)
    ref = None
    for cfg in gs.RASTER_CONFIGS:
        ctx.set_raster(*cfg)
        got = [t.clone() for t in ctx.render_mono(ds, dom, cam)]
        ctx.check_ok()
        if ref is None:
            ref = got
        else:
            assert all(torch.equal(a, b) for a, b in zip(ref, got)), cfg


def test_ellipsoid_bounds_enclose_oracle_boxes(gs, orc):
    scene, cam, dom, aff = _case("small")
    ctx = make_ctx(gs, scene, cam, keep_intermediates=True)
    ctx.render_two_pass(gs.DeviceScene(scene), dom, aff, cam)
    ctx.check_ok()
    for eye in (0, 1):
        bounds, _ = ctx.buffer(gs.BUF_BOUNDS, torch.float32, (-1, 4), eye=eye)
        rects, _ = ctx.buffer(gs.BUF_RECTS, torch.int16, (-1, 4), eye=eye)
        counts, _ = ctx.buffer(gs.BUF_COUNTS, torch.int32, None, eye=eye)
        b = bounds[: scene.n].cpu().numpy()
        r = rects[: scene.n].cpu().numpy().astype(np.int32)
        c = counts[: scene.n].cpu().numpy()
        sp = orc.prepare(scene, [dom, aff][eye], cam)
        vis = np.array([s.visible for s in sp], bool)
        assert all(s.prim == 1 for s in sp if s.visible)
        nz = c > 0
        assert nz.sum() > 0.5 * vis.sum()
        assert not (nz & ~vis).any(), "GPU bins an ellipsoid the oracle culls"
        for i in np.where(nz)[0][:3000]:
            rr, cc = orc.tile_rect(b[i], cam.width, cam.height)
            assert cc == c[i] and list(rr) == list(r[i]), i
            bx = sp[i].box
            assert b[i, 0] <= bx[0] + 1e-3 and b[i, 1] >= bx[1] - 1e-3, i
            assert b[i, 2] <= bx[2] + 1e-3 and b[i, 3] >= bx[3] - 1e-3, i


@pytest.fixture(scope="module")
def stereo_ell(gs):
    scene, cam, dom, aff = _case("small")
    ctx = make_ctx(gs, scene, cam)
    ds = gs.DeviceScene(scene)
    out = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2)
    ctx.check_ok()
    return {"scene": scene, "cam": cam, "dom": dom, "aff": aff, "ds": ds, "out": out}


def test_ellipsoid_roi_tiles_equal_the_full_affiliated_render(gs, stereo_ell):
    s = stereo_ell
    ctx = make_ctx(gs, s["scene"], s["cam"])
    tp = ctx.render_two_pass(s["ds"], s["dom"], s["aff"], s["cam"])
    ctx.check_ok()
    o = s["out"]
    rend = (o["cls_aff"] & gs.CLS_RENDER) > 0
    assert rend.any()
    assert torch.equal(o["rgb_aff"][:, rend], tp["rgb_aff"][:, rend])
    assert torch.equal(o["rgb_dom"], tp["rgb_dom"])


def test_ellipsoid_stereo_end_to_end_against_oracle(stereo_ell, orc):
    s = stereo_ell
    ref = orc.stereo(s["scene"], s["dom"], s["aff"], s["cam"], gap_thresh=2)
    o = s["out"]
    same = o["cls_aff"].cpu().numpy() == ref["cls"]
    assert same.mean() > 0.99
    assert np.array_equal(ref["widths"], o["edge_widths"].cpu().numpy())
    err = np.abs(_np(o["rgb_aff"]) - ref["rgb_aff"])[:, same]
    assert np.quantile(err, 0.999) <= RGB_TOL


def test_ellipsoid_graph_replay_and_primitive_switch(gs):
    """The primitive is part of a call's configuration: alternating surfel and
    ellipsoid calls on one context (graphs on) each give their own image."""
    scene, cam, dom, _ = synth.workload_small()
    ell = synth.to_ellipsoids(scene, 0.3)
    ctx = make_ctx(gs, scene, cam)
    d2, d3 = gs.DeviceScene(scene), gs.DeviceScene(ell)
    first = {}
    for k in range(4):
        for name, ds in (("2d", d2), ("3d", d3)):
            img = ctx.render_mono(ds, dom, cam)[0].clone()
            ctx.check_ok()
            if name in first:
                assert torch.equal(first[name], img), (name, k)
            else:
                first[name] = img
    assert not torch.equal(first["2d"], first["3d"])


def test_ellipsoid_argument_errors(gs):
    scene, cam, dom, _ = synth.workload_small()
    ell = synth.to_ellipsoids(scene)
    with pytest.raises(ValueError):
        gs.DeviceScene(synth.Scene(ell.pos, ell.quat, scene.scale, ell.opacity, ell.sh, ell.sh_degree, 1))
    ctx = make_ctx(gs, scene, cam)
    ds = gs.DeviceScene(ell)
    ds.c.primitive = 2
    with pytest.raises(gs.GsError):
        ctx.render_mono(ds, dom, cam)
