"""GPU SSIM (gs_ssim) against the FP64 oracle: random and rendered images at
sizes that span several 32-pixel tiles with ragged tails, images smaller than
the window, one to three channels; the identity at full size. The GPU filters in
float32 (the variances are differences of second moments, as in the evaluation
code the convention comes from), so the mean agrees within 1e-4."""
import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import gs as gsmod
    return gsmod


@pytest.fixture(scope="module")
def metrics():
    from oracle import metrics as M
    return M


@pytest.mark.parametrize("shape,noise", [((3, 100, 77), 0.05), ((3, 5, 7), 0.1), ((1, 64, 64), 0.02),
                                         ((2, 33, 129), 0.2), ((3, 203, 321), 0.01)])
def test_ssim_matches_oracle(gs, metrics, shape, noise):
    rng = np.random.default_rng(sum(shape))
    a = rng.random(shape)
    b = np.clip(a + noise * rng.standard_normal(shape), 0.0, 1.0)
    ta = torch.tensor(a, dtype=torch.float32, device="cuda")
    tb = torch.tensor(b, dtype=torch.float32, device="cuda")
    ctx = gs.Context(16, 512, 512, max_instances=1 << 12)
    g = float(ctx.ssim(ta, tb))
    o = metrics.ssim(ta.double().cpu().numpy(), tb.double().cpu().numpy())
    assert abs(g - o) <= TOL, (g, o)


def test_ssim_of_rendered_images(gs, metrics):
    scene, cam, dom, aff = synth.workload_small()
    ds = gs.DeviceScene(scene)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 22)
    st = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2, roi=gs.roi_params(enable_center=0))
    tp = ctx.render_two_pass(ds, dom, aff, cam)
    a, b = st["rgb_aff"].contiguous(), tp["rgb_aff"].contiguous()
    g = float(ctx.ssim(a, b))
    o = metrics.ssim(a.double().cpu().numpy(), b.double().cpu().numpy())
    assert abs(g - o) <= TOL and o < 1.0, (g, o)


def test_ssim_identity_at_full_size(gs):
    rng = np.random.default_rng(7)
    x = torch.tensor(rng.random((3, 1200, 1600)), dtype=torch.float32, device="cuda")
    ctx = gs.Context(16, 1600, 1200, max_instances=1 << 12)
    assert abs(float(ctx.ssim(x, x)) - 1.0) <= 1e-5


def test_ssim_argument_errors(gs):
    ctx = gs.Context(16, 64, 64, max_instances=1 << 12)
    x = torch.zeros(3, 65, 64, device="cuda")
    with pytest.raises(gs.GsError):
        ctx.ssim(x, x)  # taller than the context
    y = torch.zeros(4, 8, 8, device="cuda")
    with pytest.raises(gs.GsError):
        ctx.ssim(y, y)  # four channels
