"""gs_warp_noalloc, the allocation-free forward warp, against the warp stage of
gs_render_stereo on the same dominant render.

Both run the same FP32 arithmetic, so the hole masks and winning source pixels
must agree exactly; colours within the RGB tolerance of the parity tests
(2e-4) and depths within the warp test's 2e-6 relative (+inf background samples
on the same pixels). Two calls run back to back with different poses and frame
sizes, so the second also shows that no state of the first leaks through the
shared static scratch. This file is collected last so that it also runs after
every other test in the same process.
"""
import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RGB_TOL = 2e-4
WARP_DEPTH_RTOL = 2e-6
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs as gsmod
    return gsmod


def _cases():
    scene, cam, dom, aff = synth.workload_small()
    cam2 = synth.centred_camera(250, 171, 280.0)
    dom2, aff2 = synth.eye_pair(synth.look_at([0.25, -0.1, 0.1], [0.0, 0.0, 3.0]))
    return scene, [(cam, dom, aff), (cam2, dom2, aff2)]


def test_noalloc_warp_matches_stereo_warp_two_calls(gs):
    scene, cases = _cases()
    ctx = gs.Context(scene.n, 256, 192, max_instances=1 << 22)
    ds = gs.DeviceScene(scene)
    for cam, dom, aff in cases:
        H, W = cam.height, cam.width
        out = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2)
        ctx.check_ok()
        warp, _ = ctx.buffer(gs.BUF_WARP, torch.int64, None)
        wdep, _ = ctx.buffer(gs.BUF_WARP_DEPTH, torch.float32, None)
        ref_key = warp[: H * W].cpu().numpy().view(np.uint64).reshape(H, W)
        ref_dep = wdep[: H * W].cpu().numpy().reshape(H, W)
        torch.cuda.synchronize()

        rgb_w = torch.full((3, H, W), -1.0, device="cuda")
        dep_w = torch.full((H, W), -1.0, device="cuda")
        hole = torch.full((H, W), 7, dtype=torch.uint8, device="cuda")
        gs.warp_noalloc(out["rgb_dom"], out["depth_dom"], out["trans_dom"], dom, aff, cam, rgb_w, dep_w, hole)
        torch.cuda.synchronize()

        ref_hole = ref_key == EMPTY
        assert 0.0 < ref_hole.mean() < 0.5
        assert np.array_equal(hole.cpu().numpy().astype(bool), ref_hole)
        src = (ref_key & np.uint64(0xFFFFFFFF)).astype(np.int64)
        rgb_dom = out["rgb_dom"].cpu().numpy().reshape(3, -1)
        want_rgb = np.where(ref_hole[None], 0.0, rgb_dom[:, np.where(ref_hole, 0, src).ravel()].reshape(3, H, W))
        np.testing.assert_allclose(rgb_w.cpu().numpy(), want_rgb, rtol=0, atol=RGB_TOL)
        got_dep = dep_w.cpu().numpy()
        valid = ~ref_hole
        assert np.all(got_dep[ref_hole] == 0.0)
        assert np.array_equal(np.isinf(got_dep[valid]), np.isinf(ref_dep[valid]))
        fin = valid & np.isfinite(ref_dep)
        np.testing.assert_allclose(got_dep[fin], ref_dep[fin], rtol=WARP_DEPTH_RTOL)


def test_noalloc_warp_rejects_frames_above_its_scratch(gs):
    cam = synth.centred_camera(2049, 2048, 1000.0)
    dom, aff = synth.eye_pair(synth.identity_pose())
    H, W = cam.height, cam.width
    rgb = torch.zeros(3, H, W, device="cuda")
    plane = torch.zeros(H, W, device="cuda")
    with pytest.raises(gs.GsError) as e:
        gs.warp_noalloc(rgb, plane, plane, dom, aff, cam, rgb)
    assert e.value.status == gs.GS_ERR_CAPACITY
