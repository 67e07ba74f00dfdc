"""The C ABI library builds, loads without a GPU and exports every function that
include/gs.h declares; host-side argument checks that need no device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[a-z_0-9]+\s+)*\**\s*(gs_[a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def gslib():
    from paper_2609_30741_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("gs_render_mono", "gs_render_stereo", "gs_render_two_pass", "gs_context_create",
                     "gs_workspace_size", "gs_context_check", "gs_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(gslib):
    missing = [n for n in declared_functions() if not hasattr(gslib, n)]
    assert not missing, missing


def test_binding_covers_the_header(gslib):
    from paper_2609_30741_gb300 import gs
    assert set(gs.EXPORTS) <= set(declared_functions())
    gs.lib()  # loads and sets every prototype


def test_status_strings(gslib):
    from paper_2609_30741_gb300 import gs
    assert gs.status_str(gs.GS_OK) == "ok"
    assert "capacity" in gs.status_str(gs.GS_ERR_CAPACITY)


def test_workspace_size_and_limit_checks(gslib):
    from paper_2609_30741_gb300 import gs
    lim = gs.Limits(20000, 256, 192, 1 << 20, 1024, 0)
    n = C.c_size_t()
    assert gs.lib().gs_workspace_size(C.byref(lim), C.byref(n)) == gs.GS_OK
    # records for two eyes and one surfel id per instance at least
    assert n.value > 2 * 20000 * 64 + (1 << 20) * 4
    bad = gs.Limits(20000, 256, 192, 1 << 31, 1024, 0)  # instances must stay below 2^31
    assert gs.lib().gs_workspace_size(C.byref(bad), C.byref(n)) == gs.GS_ERR_BAD_ARG
    bad = gs.Limits(20000, 0, 192, 1 << 20, 1024, 0)
    assert gs.lib().gs_workspace_size(C.byref(bad), C.byref(n)) == gs.GS_ERR_BAD_ARG
    bad = gs.Limits(20000, 8200, 192, 1 << 20, 1024, 0)  # wider than the binning's shared memory allows
    assert gs.lib().gs_workspace_size(C.byref(bad), C.byref(n)) == gs.GS_ERR_BAD_ARG


def test_context_create_rejects_bad_workspace(gslib):
    from paper_2609_30741_gb300 import gs
    lim = gs.Limits(100, 64, 64, 1 << 16, 64, 0)
    h = C.c_void_p()
    # a NULL or misaligned workspace is rejected before any device call
    assert gs.lib().gs_context_create(C.byref(h), C.byref(lim), None, 1 << 20, None) == gs.GS_ERR_BAD_ARG
    assert gs.lib().gs_context_create(C.byref(h), C.byref(lim), C.c_void_p(0x1001), 1 << 30, None) == gs.GS_ERR_BAD_ARG
    assert gs.lib().gs_context_create(C.byref(h), C.byref(lim), C.c_void_p(0x100000), 16, None) == gs.GS_ERR_WORKSPACE


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_30741_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "oracle.h" not in txt, f


def test_warp_noalloc_rejects_mis_sized_tensors_before_any_launch():
    """gs_warp_noalloc takes plain pointers, so the binding checks element counts,
    dtypes and devices first: a short, mistyped or misplaced tensor raises
    ValueError and nothing reaches the device (CPU tensors stand in here)."""
    import torch
    from paper_2609_30741_gb300 import gs, synth
    cam = synth.centred_camera(40, 24, 50.0)
    H, W = cam.height, cam.width
    cpu = torch.device("cpu")
    rgb, plane = torch.zeros(3, H, W), torch.zeros(H, W)
    hole = torch.zeros(H, W, dtype=torch.uint8)
    gs.check_warp_noalloc_args(cam, cpu, rgb, plane, plane, rgb.clone(), plane.clone(), hole)  # well-formed
    bad = [
        dict(rgb_warp=torch.zeros(3, H, W - 1)),                # one column short
        dict(depth_warp=torch.zeros(H * W + 1)),                # one element long
        dict(hole=torch.zeros(H, W, dtype=torch.int32)),        # wrong dtype
        dict(trans_dom=torch.zeros(H, W, dtype=torch.float64)),
        dict(rgb_dom=torch.zeros(3, W, H).transpose(1, 2)),     # not contiguous
        dict(depth_dom=torch.zeros(H, W, device="meta")),       # another device
        dict(rgb_warp=None),                                    # a required output missing
    ]
    for change in bad:
        args = dict(rgb_dom=rgb, depth_dom=plane, trans_dom=plane, rgb_warp=rgb.clone(), depth_warp=plane.clone(),
                    hole=hole)
        args.update(change)
        with pytest.raises(ValueError):
            gs.check_warp_noalloc_args(cam, cpu, **args)
    with pytest.raises(ValueError):
        gs.warp_noalloc(rgb, plane, plane, *synth.eye_pair(synth.identity_pose()), cam, rgb.clone())


def test_workspace_follows_paths_and_per_eye_capacity(gslib):
    """The workspace holds only what the served paths use: leaving the stereo
    path out drops its per-pixel buffers (warp keys 8, warped depth 4, classes
    1, component labels 4, root slots 4, centre-hole list 4 = 25 B per pixel),
    the repair path its features and fill (16 + 12 B per pixel), the reuse path
    its strip image (12 B per pixel); a smaller affiliated-eye instance capacity
    shrinks that eye's instance, span and band-list buffers."""
    from paper_2609_30741_gb300 import gs

    def size(**kw):
        args = dict(max_surfels=20000, max_width=320, max_height=240, max_instances=1 << 20, max_rects=1024,
                    keep_intermediates=0, min_tile=16, host_outputs=0, max_instances_aff=0, paths=0)
        args.update(kw)
        n = C.c_size_t()
        st = gs.lib().gs_workspace_size(C.byref(gs.Limits(*args.values())), C.byref(n))
        return st, n.value

    P = 320 * 240
    full = size()[1]
    assert size(paths=gs.PATH_ALL)[1] == full
    no_stereo = size(paths=gs.PATH_ALL & ~gs.PATH_STEREO)[1]
    assert abs((full - no_stereo) - 25 * P) <= 256 * 7
    no_repair = size(paths=gs.PATH_ALL & ~gs.PATH_REPAIR)[1]
    assert abs((full - no_repair) - 28 * P) <= 256 * 3
    no_reuse = size(paths=gs.PATH_ALL & ~gs.PATH_REUSE)[1]
    assert abs((full - no_reuse) - 12 * P) <= 256 * 2
    small_aff = size(max_instances_aff=1 << 16)[1]
    # per instance: surfel id 4 B + span 8 B; band entries (12 B) are capped at
    # the smaller of the span capacity and 8 per surfel
    band = 12 * (min(1 << 20, 8 * 20000) - min(1 << 16, 8 * 20000))
    assert abs((full - small_aff) - 12 * ((1 << 20) - (1 << 16)) - band) <= 256 * 4
    assert size(paths=16)[0] == gs.GS_ERR_BAD_ARG
    assert size(max_instances_aff=-1)[0] == gs.GS_ERR_BAD_ARG
