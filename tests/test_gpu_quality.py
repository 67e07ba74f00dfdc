"""Where the method's error against the full render comes from on the 500k-surfel
object workload (1600x1200, SH degree 3): the reprojected pixels carry the
dominant eye's view-dependent colour (Sec. 3.4: a pixel is warped with its
colour, Sec. 4.6 names view-dependent effects as the method's limit). With the SH
bands above degree 0 zeroed (same geometry, opacities and poses) the same
pipeline must clear the DTU quality floor, and the warped pixels must carry most
of the squared error of the SH3 scene."""
import math

import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PSNR_GATE_DTU = 33.40  # two-pass DTU PSNR (Table 2) + 4.57 dB headroom


def _psnr(a, b):
    mse = torch.mean((a - b) ** 2).item()
    return 10 * math.log10(1.0 / max(mse, 1e-20))


@pytest.fixture(scope="module")
def frames():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs
    scene, cam, _, _ = synth.workload_object()
    sc0 = synth.Scene(scene.pos, scene.quat, scene.scale, scene.opacity, scene.sh.copy(), scene.sh_degree,
                      scene.primitive)
    sc0.sh[:, 1:, :] = 0.0
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 26)
    rows = []
    for name, sc in (("sh3", scene), ("sh0", sc0)):
        ds = gs.DeviceScene(sc)
        for k in (0, 3, 7):
            d, a = synth.eye_pair(synth.arc_poses()[k])
            o = {kk: v.clone() for kk, v in ctx.render_stereo(ds, d, a, cam, gap_thresh=2).items()}
            full = ctx.render_two_pass(ds, d, a, cam)["rgb_aff"].clone()
            ctx.check_ok()
            e2 = ((o["rgb_aff"] - full) ** 2).sum(0)
            c = o["cls_aff"]
            warped = ((c & gs.CLS_HOLE) == 0) & ((c & gs.CLS_RENDER) == 0)
            rend = (c & gs.CLS_RENDER) > 0
            rows.append(dict(scene=name, pose=k, psnr=_psnr(o["rgb_aff"], full),
                             warped_share=float(e2[warped].sum() / max(float(e2.sum()), 1e-30)),
                             roi_err=float(e2[rend].max()) if bool(rend.any()) else 0.0))
    for r in rows:
        print(r)
    return rows


def test_view_independent_colour_clears_the_quality_floor(frames):
    sh0 = [r for r in frames if r["scene"] == "sh0"]
    sh3 = [r for r in frames if r["scene"] == "sh3"]
    assert min(r["psnr"] for r in sh0) >= PSNR_GATE_DTU
    for a, b in zip(sh0, sh3):
        assert a["psnr"] >= b["psnr"] + 8.0, (a, b)


def test_warped_pixels_carry_the_view_dependent_error(frames):
    for r in frames:
        assert r["roi_err"] == 0.0, r  # re-rendered pixels are the full render's
        if r["scene"] == "sh3":
            assert r["warped_share"] >= 0.7, r
