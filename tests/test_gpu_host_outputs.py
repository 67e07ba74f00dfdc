"""gs_render_stereo_host: the method with both eyes' RGB images delivered to
page-locked host memory. The images equal gs_render_stereo's device outputs bit
for bit, in direct launches and graph replays (the host copies are nodes of the
captured graph), for a new pose on every call and with depth_mode 2; pageable
host memory, device memory and a context without host outputs are rejected."""
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


@pytest.fixture(scope="module")
def setup(gs):
    scene = synth.scene_object_ground(1401, n=60_000)
    cam = synth.centred_camera(480, 360, 480.0)
    pairs = [synth.eye_pair(p) for p in synth.arc_poses()[:4]]
    return scene, cam, pairs, gs.DeviceScene(scene)


def _host(cam):
    return [torch.empty(3, cam.height, cam.width, dtype=torch.float32).pin_memory() for _ in range(2)]


@pytest.mark.parametrize("depth_mode", [0, 2])
def test_host_images_equal_device_outputs(gs, setup, depth_mode):
    scene, cam, pairs, ds = setup
    a = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 23, host_outputs=True)
    b = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 23)
    roi = gs.roi_params(depth_mode=depth_mode)
    hd, ha = _host(cam)
    for k, (d, f) in enumerate(pairs + pairs[::-1]):  # direct, capture, replays with new poses
        hd.fill_(-1.0)
        ha.fill_(-1.0)
        a.render_stereo_host(ds, d, f, cam, hd, ha, gap_thresh=2, roi=roi)
        a.check_ok()  # synchronises the stream: the host images are complete
        ref = b.render_stereo(ds, d, f, cam, gap_thresh=2, roi=roi)
        b.check_ok()
        assert torch.equal(hd, ref["rgb_dom"].cpu()), k
        assert torch.equal(ha, ref["rgb_aff"].cpu()), k


def test_host_outputs_argument_errors(gs, setup):
    scene, cam, pairs, ds = setup
    d, f = pairs[0]
    a = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 23, host_outputs=True)
    pageable = [torch.empty(3, cam.height, cam.width, dtype=torch.float32) for _ in range(2)]
    with pytest.raises(gs.GsError):
        a.render_stereo_host(ds, d, f, cam, *pageable)
    hd, ha = _host(cam)
    with pytest.raises(gs.GsError):  # sized without host outputs
        gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 23).render_stereo_host(ds, d, f, cam, hd, ha)
    with pytest.raises(ValueError):  # device memory is not a host image
        a.render_stereo_host(ds, d, f, cam, hd.cuda(), ha)
    a.render_stereo_host(ds, d, f, cam, hd, ha)
    a.check_ok()
