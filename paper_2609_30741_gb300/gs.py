"""Python binding of the C ABI in include/gs.h (ctypes; argument marshalling only).

Every stage of the pipeline runs in libgs.so's CUDA kernels. PyTorch supplies the
device memory (scene, outputs and the context workspace) and the CUDA stream.
Importing this module loads the in-tree libgs.so and fails loudly when it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgs.so")

GS_OK, GS_ERR_BAD_ARG, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_CUDA, GS_ERR_WORKSPACE, GS_ERR_NOT_LOADED = range(7)
(BUF_RECORDS, BUF_RECTS, BUF_BOUNDS, BUF_COUNTS, BUF_DEPTH_ORDER, BUF_INST_KEYS, BUF_INST_VALS, BUF_RANGES,
 BUF_WARP, BUF_TILE_MASK, BUF_DEPTH_RANGE, BUF_STRIPS, BUF_WARP_DEPTH, BUF_PAIRS, BUF_BIN_COUNTS) = range(15)
BUF_EYE1 = 0x100
CLS_HOLE, CLS_GAP, CLS_CENTRE, CLS_STRIP, CLS_RENDER, CLS_NET = 1, 2, 4, 8, 16, 32
PATH_MONO, PATH_STEREO, PATH_REUSE, PATH_REPAIR, PATH_ALL = 1, 2, 4, 8, 15


class GsError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        detail = ""
        if status == GS_ERR_CUDA:
            detail = f" [{lib().gs_last_cuda_error().decode()}]"
        super().__init__(f"{what}: {status_str(status)} ({status}){detail}")


class Scene(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("n", C.c_int), ("sh_degree", C.c_int), ("primitive", C.c_int)]


class Pose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int), ("height", C.c_int)]


class RoiParams(C.Structure):
    _fields_ = [("margin", C.c_int), ("samples_per_edge", C.c_int), ("enable_center", C.c_int),
                ("depth_mode", C.c_int), ("d_min", C.c_float), ("d_max", C.c_float),
                ("repair_mode", C.c_int), ("gate_tau", C.c_float)]


class Outputs(C.Structure):
    _fields_ = [("rgb_dom", C.c_void_p), ("depth_dom", C.c_void_p), ("trans_dom", C.c_void_p),
                ("rgb_aff", C.c_void_p), ("cls_aff", C.c_void_p), ("roi_rects", C.c_void_p),
                ("roi_count", C.c_void_p), ("edge_widths", C.c_void_p)]


class Limits(C.Structure):
    _fields_ = [("max_surfels", C.c_int), ("max_width", C.c_int), ("max_height", C.c_int),
                ("max_instances", C.c_int64), ("max_rects", C.c_int), ("keep_intermediates", C.c_int),
                ("min_tile", C.c_int), ("host_outputs", C.c_int), ("max_instances_aff", C.c_int64),
                ("paths", C.c_int)]


class Usage(C.Structure):
    """Work counts of a context's last call (gs_usage), per eye."""
    _fields_ = [("binned", C.c_int64 * 2), ("instances", C.c_int64 * 2), ("spans", C.c_int64 * 2),
                ("band_entries", C.c_int64 * 2)]

    def asdict(self):
        return {k: [int(v) for v in getattr(self, k)] for k, _ in self._fields_}


class RasterConfig(C.Structure):
    """Rasterizer tile edge, pixels per thread and records per shared-memory stage."""
    _fields_ = [("tile", C.c_int), ("pix", C.c_int), ("batch", C.c_int)]

    def astuple(self):
        return (self.tile, self.pix, self.batch)


class Frame(C.Structure):
    """One frame of a batch (gs_frame)."""
    _fields_ = [("scene", C.c_void_p), ("pose_dom", Pose), ("pose_aff", Pose), ("intr", Intrinsics),
                ("out", Outputs)]


class MonoFrame(C.Structure):
    """One eye of gs_render_mono_batch (gs_mono_frame)."""
    _fields_ = [("scene", C.c_void_p), ("pose", Pose), ("intr", Intrinsics), ("bg", C.c_float * 3),
                ("rgb", C.c_void_p), ("depth", C.c_void_p), ("trans", C.c_void_p)]


class TuneResult(C.Structure):
    _fields_ = [("rc", RasterConfig), ("ms", C.c_float)]


# every valid (tile, pix, batch): the autotuner's search space
RASTER_CONFIGS = [(t, p, b) for t, ps in ((8, (1, 2)), (16, (2, 4)), (32, (2, 4, 8))) for p in ps
                  for b in (32, 64, 128, 256)]


class RepairBatch(C.Structure):
    _fields_ = [("feat", C.c_void_p), ("target", C.c_void_p), ("plain", C.c_void_p), ("frames", C.c_int),
                ("width", C.c_int), ("height", C.c_int), ("tiles", C.c_void_p), ("n_tiles", C.c_int),
                ("scratch", C.c_void_p)]


class AdamW(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float), ("gate_weight", C.c_float)]


EXPORTS = {
    "gs_status_str": (C.c_char_p, [C.c_int]),
    "gs_kernel_launches": (C.c_ulonglong, []),
    "gs_last_cuda_error": (C.c_char_p, []),
    "gs_workspace_size": (C.c_int, [C.POINTER(Limits), C.POINTER(C.c_size_t)]),
    "gs_set_programmatic_launch": (None, [C.c_int]),
    "gs_programmatic_launch": (C.c_int, []),
    "gs_context_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Limits), C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs_context_destroy": (C.c_int, [C.c_void_p]),
    "gs_context_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gs_context_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "gs_context_usage": (C.c_int, [C.c_void_p, C.POINTER(Usage)]),
    "gs_context_set_counting": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_context_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_context_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_context_set_raster": (C.c_int, [C.c_void_p, C.POINTER(RasterConfig)]),
    "gs_context_set_raster_roi": (C.c_int, [C.c_void_p, C.POINTER(RasterConfig)]),
    "gs_context_get_raster_roi": (C.c_int, [C.c_void_p, C.POINTER(RasterConfig), C.POINTER(C.c_int)]),
    "gs_context_get_raster": (C.c_int, [C.c_void_p, C.POINTER(RasterConfig)]),
    "gs_context_stage_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]),
    "gs_context_buffer": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t),
                                    C.POINTER(C.c_int64)]),
    "gs_render_mono": (C.c_int, [C.c_void_p, C.POINTER(Scene), C.POINTER(Pose), C.POINTER(Intrinsics),
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_render_stereo": (C.c_int, [C.c_void_p, C.POINTER(Scene), C.POINTER(Pose), C.POINTER(Pose),
                                   C.POINTER(Intrinsics), C.c_int, C.POINTER(RoiParams), C.POINTER(Outputs)]),
    "gs_render_stereo_host": (C.c_int, [C.c_void_p, C.POINTER(Scene), C.POINTER(Pose), C.POINTER(Pose),
                                        C.POINTER(Intrinsics), C.c_int, C.POINTER(RoiParams), C.c_void_p,
                                        C.c_void_p]),
    "gs_render_two_pass": (C.c_int, [C.c_void_p, C.POINTER(Scene), C.POINTER(Pose), C.POINTER(Pose),
                                     C.POINTER(Intrinsics), C.POINTER(Outputs)]),
    "gs_warp_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Pose), C.POINTER(Pose),
                                  C.POINTER(Intrinsics), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "gs_batch_destroy": (C.c_int, [C.c_void_p]),
    "gs_batch_set_raster": (C.c_int, [C.c_void_p, C.POINTER(RasterConfig)]),
    "gs_batch_get_raster": (C.c_int, [C.c_void_p, C.POINTER(RasterConfig)]),
    "gs_batch_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_batch_set_counting": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_batch_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_batch_stage_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]),
    "gs_batch_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "gs_render_stereo_batch": (C.c_int, [C.c_void_p, C.POINTER(Frame), C.c_int, C.c_int, C.POINTER(RoiParams)]),
    "gs_render_two_pass_batch": (C.c_int, [C.c_void_p, C.POINTER(Frame), C.c_int]),
    "gs_render_mono_batch": (C.c_int, [C.c_void_p, C.POINTER(MonoFrame), C.c_int]),
    "gs_autotune_batch": (C.c_int, [C.c_void_p, C.POINTER(Frame), C.c_int, C.c_int, C.POINTER(RoiParams), C.c_int,
                                    C.c_int, C.POINTER(TuneResult), C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(RasterConfig), C.POINTER(C.c_float)]),
    "gs_autotune_stereo": (C.c_int, [C.c_void_p, C.POINTER(Scene), C.POINTER(Pose), C.POINTER(Pose),
                                     C.POINTER(Intrinsics), C.c_int, C.POINTER(RoiParams), C.POINTER(Outputs), C.c_int,
                                     C.c_int, C.POINTER(TuneResult), C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(RasterConfig), C.POINTER(C.c_float)]),
    "gs_tune_cache_save": (C.c_int, [C.c_char_p]),
    "gs_tune_cache_load": (C.c_int, [C.c_char_p]),
    "gs_tune_cache_clear": (C.c_int, []),
    "gs_tune_cache_size": (C.c_int, [C.POINTER(C.c_int)]),
    "gs_tune_cache_put": (C.c_int, [C.c_char_p, C.POINTER(RasterConfig), C.c_float]),
    "gs_tune_cache_get": (C.c_int, [C.c_char_p, C.POINTER(RasterConfig), C.POINTER(C.c_float)]),
    "gs_ssim": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "gs_centre_rois": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "gs_repair_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "gs_repair_read": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "gs_repair_steps": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "gs_repair_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "gs_repair_features": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "gs_repair_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                  C.c_void_p, C.c_void_p, C.c_int]),
    "gs_repair_calibrate_fp8": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "gs_repair_read_fp8_scales": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gs_repair_train_scratch_size": (C.c_int, [C.c_int, C.POINTER(C.c_size_t)]),
    "gs_repair_train_step": (C.c_int, [C.c_void_p, C.POINTER(RepairBatch), C.POINTER(AdamW), C.c_void_p]),
}

REPAIR_PARAMS = 39908

WARP_NOALLOC_MAX_PIXELS = 1 << 22

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2609_30741_gb300.build.build() "
                              "(there is no CPU fallback)")
        lib_ = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(lib_, name)
            f.restype = res
            f.argtypes = args
        _lib = lib_
    return _lib


def kernel_launches() -> int:
    """Kernels libgs.so has enqueued since it was loaded."""
    return int(lib().gs_kernel_launches())


def set_programmatic_launch(on: bool):
    """Programmatic dependent launch of the library's kernels (default on)."""
    lib().gs_set_programmatic_launch(int(bool(on)))


def programmatic_launch() -> bool:
    return bool(lib().gs_programmatic_launch())


def status_str(s: int) -> str:
    return lib().gs_status_str(int(s)).decode()


def _check(s, what):
    if s != GS_OK:
        raise GsError(s, what)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def pose_struct(pose) -> Pose:
    import numpy as np
    return Pose((C.c_double * 9)(*np.asarray(pose.R, np.float64).ravel()),
                (C.c_double * 3)(*np.asarray(pose.t, np.float64).ravel()))


def intr_struct(cam) -> Intrinsics:
    return Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)


def roi_params(margin=32, samples_per_edge=32, enable_center=1, depth_mode=0, d_min=0.0, d_max=0.0,
               repair_mode=0, gate_tau=0.5) -> RoiParams:
    return RoiParams(margin, samples_per_edge, enable_center, depth_mode, d_min, d_max, repair_mode, gate_tau)


class DeviceScene:
    """Primitive attributes resident on the GPU (torch tensors) + the C struct.
    `scene.primitive` (default 0) selects 2D surfels (scale [n, 2]) or 3D
    ellipsoids (scale [n, 4]: s_x, s_y, s_z, pad)."""

    def __init__(self, scene, device="cuda"):
        def t(a):
            return torch.as_tensor(a).to(device=device, dtype=torch.float32).contiguous()
        self.pos, self.quat, self.scale = t(scene.pos), t(scene.quat), t(scene.scale)
        self.opacity, self.sh = t(scene.opacity), t(scene.sh)
        self.n, self.sh_degree = int(scene.n), int(scene.sh_degree)
        self.primitive = int(getattr(scene, "primitive", 0))
        want = 4 if self.primitive == 1 else 2
        if self.n and tuple(self.scale.shape) != (self.n, want):
            raise ValueError(f"scale must be [{self.n}, {want}] for primitive {self.primitive}")
        self.c = Scene(self.pos.data_ptr(), self.quat.data_ptr(), self.scale.data_ptr(),
                       self.opacity.data_ptr(), self.sh.data_ptr(), self.n, self.sh_degree, self.primitive)

    def nbytes(self):
        return sum(x.numel() * 4 for x in (self.pos, self.quat, self.scale, self.opacity, self.sh))


class Context:
    """A renderer context: owns its workspace tensor, runs on a torch stream."""

    def __init__(self, max_surfels, max_width, max_height, max_instances=1 << 24, max_rects=1 << 16,
                 keep_intermediates=False, device="cuda", stream=None, min_tile=16, host_outputs=False,
                 max_instances_aff=0, paths=0):
        """max_instances_aff: instance capacity of the affiliated eye (0: as the
        dominant eye); paths: PATH_* bits of the entry points the context serves
        (0: all), which leaves other paths' buffers out of the workspace."""
        self.lim = Limits(int(max_surfels), int(max_width), int(max_height), int(max_instances),
                          int(max_rects), int(bool(keep_intermediates)), int(min_tile), int(bool(host_outputs)),
                          int(max_instances_aff), int(paths))
        nbytes = C.c_size_t()
        _check(lib().gs_workspace_size(C.byref(self.lim), C.byref(nbytes)), "gs_workspace_size")
        self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(lib().gs_context_create(C.byref(h), C.byref(self.lim), C.c_void_p(base + off),
                                       C.c_size_t(nbytes.value), C.c_void_p(self.stream.cuda_stream)),
               "gs_context_create")
        self.h = h
        self.ws_offset = off

    def close(self):
        if getattr(self, "h", None):
            lib().gs_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        _check(lib().gs_context_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "gs_context_set_stream")

    def usage(self):
        """Per-eye binned surfels, instances, spans and band-list entries of the
        last call (synchronises the context's stream)."""
        u = Usage()
        _check(lib().gs_context_usage(self.h, C.byref(u)), "gs_context_usage")
        return u.asdict()

    def set_counting(self, on: bool):
        _check(lib().gs_context_set_counting(self.h, int(bool(on))), "gs_context_set_counting")

    def set_graphs(self, on: bool):
        _check(lib().gs_context_set_graphs(self.h, int(bool(on))), "gs_context_set_graphs")

    def set_raster(self, tile, pix, batch):
        rc = RasterConfig(int(tile), int(pix), int(batch))
        _check(lib().gs_context_set_raster(self.h, C.byref(rc)), "gs_context_set_raster")

    def raster(self):
        rc = RasterConfig()
        _check(lib().gs_context_get_raster(self.h, C.byref(rc)), "gs_context_get_raster")
        return rc.astuple()

    def set_raster_roi(self, config=None):
        """The ROI re-render's own (tile, pix, batch), or None to use set_raster's."""
        rc = RasterConfig(*[int(v) for v in config]) if config is not None else None
        _check(lib().gs_context_set_raster_roi(self.h, C.byref(rc) if rc is not None else None),
               "gs_context_set_raster_roi")

    def raster_roi(self):
        """(the configuration the ROI re-render uses, whether one of its own is set)"""
        rc, is_set = RasterConfig(), C.c_int()
        _check(lib().gs_context_get_raster_roi(self.h, C.byref(rc), C.byref(is_set)), "gs_context_get_raster_roi")
        return rc.astuple(), bool(is_set.value)

    def set_profiling(self, on: bool):
        _check(lib().gs_context_set_profiling(self.h, int(bool(on))), "gs_context_set_profiling")

    def stage_times(self):
        buf = (C.c_float * 16)()
        n = C.c_int()
        _check(lib().gs_context_stage_times(self.h, buf, 16, C.byref(n)), "gs_context_stage_times")
        return [buf[i] for i in range(n.value)]

    def pair_counts(self):
        """(evaluated[2], contributed[2]) pairs of the last call in counting mode."""
        v, _ = self.buffer(BUF_PAIRS, torch.int64)
        a = v[:4].cpu().tolist()
        return a[:2], a[2:]

    def check(self) -> int:
        st = C.c_int()
        _check(lib().gs_context_check(self.h, C.byref(st)), "gs_context_check")
        return st.value

    def check_ok(self):
        st = self.check()
        if st != GS_OK:
            raise GsError(st, "device status")

    def buffer(self, which, dtype, shape=None, eye=0):
        """A torch view of a workspace intermediate (see gs_buffer_id)."""
        p, nb, cnt = C.c_void_p(), C.c_size_t(), C.c_int64()
        _check(lib().gs_context_buffer(self.h, which | (BUF_EYE1 if eye else 0), C.byref(p), C.byref(nb),
                                       C.byref(cnt)), "gs_context_buffer")
        start = p.value - self.workspace.data_ptr()
        raw = self.workspace[start:start + nb.value]
        v = raw.view(dtype)
        if shape is not None:
            v = v.view(*shape)
        return v, cnt.value

    # ---------------------------------------------------------------- entry points

    def render_mono(self, scene: DeviceScene, pose, cam, bg=None, out=None):
        H, W = cam.height, cam.width
        if out is None:
            out = (torch.empty(3, H, W, device=self.device), torch.empty(H, W, device=self.device),
                   torch.empty(H, W, device=self.device))
        rgb, dep, tr = out
        bgp = (C.c_float * 3)(*bg) if bg is not None else None
        _check(lib().gs_render_mono(self.h, C.byref(scene.c), C.byref(pose_struct(pose)),
                                    C.byref(intr_struct(cam)), C.cast(bgp, C.c_void_p) if bgp else None,
                                    _ptr(rgb), _ptr(dep), _ptr(tr)), "gs_render_mono")
        return rgb, dep, tr

    def alloc_outputs(self, cam, with_cls=True):
        H, W = cam.height, cam.width
        d = self.device
        o = dict(rgb_dom=torch.empty(3, H, W, device=d), depth_dom=torch.empty(H, W, device=d),
                 trans_dom=torch.empty(H, W, device=d), rgb_aff=torch.empty(3, H, W, device=d))
        if with_cls:
            o.update(cls_aff=torch.empty(H, W, dtype=torch.uint8, device=d),
                     roi_rects=torch.empty(self.lim.max_rects, 4, dtype=torch.int32, device=d),
                     roi_count=torch.zeros(1, dtype=torch.int32, device=d),
                     edge_widths=torch.zeros(4, dtype=torch.int32, device=d))
        return o

    @staticmethod
    def _outputs_struct(o):
        return Outputs(*[(o[k].data_ptr() if o.get(k) is not None else None) for k in
                         ("rgb_dom", "depth_dom", "trans_dom", "rgb_aff", "cls_aff", "roi_rects", "roi_count",
                          "edge_widths")])

    def render_stereo(self, scene: DeviceScene, pose_dom, pose_aff, cam, gap_thresh=2, roi=None, out=None):
        if out is None:
            out = self.alloc_outputs(cam)
        roi = roi if roi is not None else roi_params()
        os_ = self._outputs_struct(out)
        _check(lib().gs_render_stereo(self.h, C.byref(scene.c), C.byref(pose_struct(pose_dom)),
                                      C.byref(pose_struct(pose_aff)), C.byref(intr_struct(cam)), int(gap_thresh),
                                      C.byref(roi), C.byref(os_)), "gs_render_stereo")
        return out

    def render_stereo_host(self, scene: DeviceScene, pose_dom, pose_aff, cam, host_rgb_dom, host_rgb_aff,
                           gap_thresh=2, roi=None):
        """gs_render_stereo_host: both eyes' RGB into page-locked host tensors
        ([3, H, W] float32, pin_memory=True); complete after the stream syncs."""
        for t in (host_rgb_dom, host_rgb_aff):
            if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous() or \
                    tuple(t.shape) != (3, cam.height, cam.width):
                raise ValueError("host images must be contiguous [3, H, W] float32 CPU tensors")
        roi = roi if roi is not None else roi_params()
        _check(lib().gs_render_stereo_host(self.h, C.byref(scene.c), C.byref(pose_struct(pose_dom)),
                                           C.byref(pose_struct(pose_aff)), C.byref(intr_struct(cam)),
                                           int(gap_thresh), C.byref(roi), C.c_void_p(host_rgb_dom.data_ptr()),
                                           C.c_void_p(host_rgb_aff.data_ptr())), "gs_render_stereo_host")

    def ssim(self, img, ref, out=None):
        """Mean SSIM of img against ref ([C, H, W] float32 CUDA tensors), as a
        device scalar tensor (gs_ssim)."""
        if img.shape != ref.shape or img.dim() != 3 or not img.is_contiguous() or not ref.is_contiguous():
            raise ValueError("ssim takes two contiguous [C, H, W] tensors of one shape")
        if out is None:
            out = torch.empty((), dtype=torch.float32, device=img.device)
        C_, H, W = img.shape
        _check(lib().gs_ssim(self.h, _ptr(img), _ptr(ref), W, H, C_, _ptr(out)), "gs_ssim")
        return out

    def centre_rois(self, cls, margin=32, tile_mask=None):
        """Centre ROIs of a [H, W] uint8 class map (gs_centre_rois): (rects
        [max_rects, 4] int32, count int32 tensor), both on the device."""
        if cls.dtype != torch.uint8 or cls.dim() != 2 or not cls.is_contiguous():
            raise ValueError("centre_rois takes a contiguous [H, W] uint8 tensor")
        H, W = cls.shape
        rects = torch.empty(self.lim.max_rects, 4, dtype=torch.int32, device=cls.device)
        count = torch.zeros(1, dtype=torch.int32, device=cls.device)
        _check(lib().gs_centre_rois(self.h, _ptr(cls), W, H, int(margin), _ptr(rects), _ptr(count),
                                    _ptr(tile_mask) if tile_mask is not None else None), "gs_centre_rois")
        return rects, count

    # ---- learned repair ----
    def repair_load(self, weights):
        import numpy as np
        w = np.ascontiguousarray(np.asarray(weights, np.float32).ravel())
        if w.size != REPAIR_PARAMS:
            raise ValueError(f"expected {REPAIR_PARAMS} parameters, got {w.size}")
        _check(lib().gs_repair_load(self.h, w.ctypes.data_as(C.c_void_p), C.c_int64(w.size)), "gs_repair_load")

    def repair_read(self, which=0):
        import numpy as np
        out = np.empty(REPAIR_PARAMS, np.float32)
        _check(lib().gs_repair_read(self.h, int(which), out.ctypes.data_as(C.c_void_p), C.c_int64(out.size)),
               "gs_repair_read")
        return out

    def repair_steps(self) -> int:
        """AdamW steps taken since the last repair_load (the bias-correction count)."""
        n = C.c_int()
        _check(lib().gs_repair_steps(self.h, C.byref(n)), "gs_repair_steps")
        return n.value

    def repair_state(self):
        """(weights, m, v, steps): everything a training checkpoint needs from the
        context."""
        return self.repair_read(0), self.repair_read(2), self.repair_read(3), self.repair_steps()

    def repair_load_state(self, weights, m, v, steps):
        import numpy as np
        arrs = [np.ascontiguousarray(np.asarray(a, np.float32).ravel()) for a in (weights, m, v)]
        if any(a.size != REPAIR_PARAMS for a in arrs):
            raise ValueError(f"repair state arrays need {REPAIR_PARAMS} floats")
        _check(lib().gs_repair_load_state(self.h, *[a.ctypes.data_as(C.c_void_p) for a in arrs],
                                          C.c_int64(REPAIR_PARAMS), int(steps)), "gs_repair_load_state")

    def repair_features(self, cam, out=None):
        """Features of the last gs_render_stereo call made with repair_mode != 0:
        (H, W, 8) bfloat16."""
        if out is None:
            out = torch.empty(cam.height, cam.width, 8, dtype=torch.bfloat16, device=self.device)
        _check(lib().gs_repair_features(self.h, cam.width, cam.height, _ptr(out)), "gs_repair_features")
        return out

    def repair_infer(self, feat, tiles, fill=None, gate=None, fp8=False):
        """feat (F, H, W, 8) bfloat16; tiles int32 tensor of frame << 24 | ty << 12 | tx."""
        F, H, W = feat.shape[0], feat.shape[1], feat.shape[2]
        if gate is None:
            gate = torch.empty(tiles.numel(), dtype=torch.float32, device=self.device)
        _check(lib().gs_repair_infer(self.h, _ptr(feat), F, W, H, _ptr(tiles), tiles.numel(), _ptr(fill),
                                     _ptr(gate), 1 if fp8 else 0), "gs_repair_infer")
        return fill, gate

    def repair_calibrate_fp8(self, feat, tiles):
        F, H, W = feat.shape[0], feat.shape[1], feat.shape[2]
        _check(lib().gs_repair_calibrate_fp8(self.h, _ptr(feat), F, W, H, _ptr(tiles), tiles.numel()),
               "gs_repair_calibrate_fp8")

    def repair_fp8_scales(self):
        """(sx, sw): the calibrated input and weight scales, (6, 32) each."""
        import numpy as np
        out = np.empty(384, np.float32)
        _check(lib().gs_repair_read_fp8_scales(self.h, out.ctypes.data_as(C.c_void_p)), "gs_repair_read_fp8_scales")
        return out[:192].reshape(6, 32), out[192:].reshape(6, 32)

    def repair_train_step(self, feat, target, plain, tiles, scratch=None, lr=1e-3, beta1=0.9, beta2=0.999,
                          eps=1e-8, weight_decay=0.0, gate_weight=0.1, want_loss=True):
        import numpy as np
        F, H, W = feat.shape[0], feat.shape[1], feat.shape[2]
        if scratch is None:
            scratch = self.repair_scratch(tiles.numel())
        b = RepairBatch(_ptr(feat), _ptr(target), _ptr(plain), F, W, H, _ptr(tiles), tiles.numel(), _ptr(scratch))
        o = AdamW(lr, beta1, beta2, eps, weight_decay, gate_weight)
        loss = np.zeros(4, np.float32)
        _check(lib().gs_repair_train_step(self.h, C.byref(b), C.byref(o),
                                          loss.ctypes.data_as(C.c_void_p) if want_loss else None),
               "gs_repair_train_step")
        return loss

    def repair_scratch(self, n_tiles):
        n = C.c_size_t()
        _check(lib().gs_repair_train_scratch_size(int(n_tiles), C.byref(n)), "gs_repair_train_scratch_size")
        return torch.empty(n.value, dtype=torch.uint8, device=self.device)

    def render_two_pass(self, scene: DeviceScene, pose_dom, pose_aff, cam, out=None):
        if out is None:
            out = self.alloc_outputs(cam, with_cls=False)
        os_ = self._outputs_struct(out)
        _check(lib().gs_render_two_pass(self.h, C.byref(scene.c), C.byref(pose_struct(pose_dom)),
                                        C.byref(pose_struct(pose_aff)), C.byref(intr_struct(cam)), C.byref(os_)),
               "gs_render_two_pass")
        return out


def _tune_out(n, res, best, ms):
    results = [(res[i].rc.astuple(), float(res[i].ms)) for i in range(n.value)]
    return best.astuple(), float(ms.value), results


def autotune_stereo(ctx, scene, pose_dom, pose_aff, cam, gap_thresh=2, roi=None, out=None, reps=5, use_cache=True,
                    two_pass=False):
    """Times every rasterizer configuration the context allows on this frame
    (gs_render_stereo, or gs_render_two_pass with two_pass=True) and keeps the
    fastest on the context: returns (best (tile, pix, batch), its median ms,
    [(config, ms), ...]); with use_cache a cached shape is applied untimed."""
    if out is None:
        out = ctx.alloc_outputs(cam)
    roi = None if two_pass else (roi if roi is not None else roi_params())
    res = (TuneResult * 32)()
    n, best, ms = C.c_int(), RasterConfig(), C.c_float()
    _check(lib().gs_autotune_stereo(ctx.h, C.byref(scene.c), C.byref(pose_struct(pose_dom)),
                                    C.byref(pose_struct(pose_aff)), C.byref(intr_struct(cam)), int(gap_thresh),
                                    C.byref(roi) if roi is not None else None,
                                    C.byref(Context._outputs_struct(out)), int(reps),
                                    int(bool(use_cache)), res, 32, C.byref(n), C.byref(best), C.byref(ms)),
           "gs_autotune_stereo")
    return _tune_out(n, res, best, ms)


class Batch:
    """Many stereo frames per call (gs_render_stereo_batch): frame f runs in
    slot f, a Context sized for it; each rasterizer pass is one persistent
    launch over all frames."""

    def __init__(self, contexts, stream=None):
        self.slots = list(contexts)
        dev = self.slots[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        arr = (C.c_void_p * len(self.slots))(*[c.h.value if isinstance(c.h, C.c_void_p) else c.h for c in self.slots])
        h = C.c_void_p()
        _check(lib().gs_batch_create(C.byref(h), arr, len(self.slots), C.c_void_p(self.stream.cuda_stream)),
               "gs_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().gs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_raster(self, tile, pix, batch):
        rc = RasterConfig(int(tile), int(pix), int(batch))
        _check(lib().gs_batch_set_raster(self.h, C.byref(rc)), "gs_batch_set_raster")

    def raster(self):
        rc = RasterConfig()
        _check(lib().gs_batch_get_raster(self.h, C.byref(rc)), "gs_batch_get_raster")
        return rc.astuple()

    def set_graphs(self, on: bool):
        _check(lib().gs_batch_set_graphs(self.h, int(bool(on))), "gs_batch_set_graphs")

    def set_counting(self, on: bool):
        _check(lib().gs_batch_set_counting(self.h, int(bool(on))), "gs_batch_set_counting")

    def set_profiling(self, on: bool):
        _check(lib().gs_batch_set_profiling(self.h, int(bool(on))), "gs_batch_set_profiling")

    def stage_times(self):
        buf = (C.c_float * 8)()
        n = C.c_int()
        _check(lib().gs_batch_stage_times(self.h, buf, 8, C.byref(n)), "gs_batch_stage_times")
        return [buf[i] for i in range(n.value)]

    def check(self) -> int:
        st = C.c_int()
        _check(lib().gs_batch_check(self.h, C.byref(st)), "gs_batch_check")
        return st.value

    def check_ok(self):
        st = self.check()
        if st != GS_OK:
            raise GsError(st, "device status")

    @staticmethod
    def frames_struct(frames):
        """frames: [(DeviceScene, pose_dom, pose_aff, cam, outputs dict)]"""
        arr = (Frame * len(frames))()
        for i, (ds, d, a, cam, out) in enumerate(frames):
            arr[i] = Frame(C.cast(C.pointer(ds.c), C.c_void_p), pose_struct(d), pose_struct(a), intr_struct(cam),
                           Context._outputs_struct(out))
        return arr

    def render_stereo(self, frames, gap_thresh=2, roi=None):
        roi = roi if roi is not None else roi_params()
        arr = self.frames_struct(frames)
        _check(lib().gs_render_stereo_batch(self.h, arr, len(frames), int(gap_thresh), C.byref(roi)),
               "gs_render_stereo_batch")

    def render_two_pass(self, frames):
        arr = self.frames_struct(frames)
        _check(lib().gs_render_two_pass_batch(self.h, arr, len(frames)), "gs_render_two_pass_batch")

    def render_mono(self, frames):
        """frames: [(DeviceScene, pose, cam, (rgb, depth, trans) tensors, bg or None)]"""
        arr = (MonoFrame * len(frames))()
        for i, (ds, pose, cam, out, bg) in enumerate(frames):
            rgb, dep, tr = out
            arr[i] = MonoFrame(C.cast(C.pointer(ds.c), C.c_void_p), pose_struct(pose), intr_struct(cam),
                               (C.c_float * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0))), rgb.data_ptr(),
                               dep.data_ptr() if dep is not None else None, tr.data_ptr() if tr is not None else None)
        _check(lib().gs_render_mono_batch(self.h, arr, len(frames)), "gs_render_mono_batch")

    def autotune(self, frames, gap_thresh=2, roi=None, reps=5, use_cache=True, two_pass=False):
        """(best (tile, pix, batch), its median ms per call, [(config, ms), ...]);
        two_pass=True tunes the two-pass comparator."""
        roi = None if two_pass else (roi if roi is not None else roi_params())
        arr = self.frames_struct(frames)
        res = (TuneResult * 32)()
        n, best, ms = C.c_int(), RasterConfig(), C.c_float()
        _check(lib().gs_autotune_batch(self.h, arr, len(frames), int(gap_thresh),
                                       C.byref(roi) if roi is not None else None, int(reps),
                                       int(bool(use_cache)), res, 32, C.byref(n), C.byref(best), C.byref(ms)),
               "gs_autotune_batch")
        return _tune_out(n, res, best, ms)


def tune_cache_save(path):
    _check(lib().gs_tune_cache_save(os.fsencode(path)), "gs_tune_cache_save")


def tune_cache_load(path):
    _check(lib().gs_tune_cache_load(os.fsencode(path)), "gs_tune_cache_load")


def tune_cache_clear():
    _check(lib().gs_tune_cache_clear(), "gs_tune_cache_clear")


def tune_cache_size() -> int:
    n = C.c_int()
    _check(lib().gs_tune_cache_size(C.byref(n)), "gs_tune_cache_size")
    return n.value


def tune_cache_put(key, config, ms):
    rc = RasterConfig(*[int(v) for v in config])
    _check(lib().gs_tune_cache_put(key.encode(), C.byref(rc), float(ms)), "gs_tune_cache_put")


def tune_cache_get(key):
    """(config, ms) or None"""
    rc, ms = RasterConfig(), C.c_float()
    s = lib().gs_tune_cache_get(key.encode(), C.byref(rc), C.byref(ms))
    if s == GS_ERR_NOT_LOADED:
        return None
    _check(s, "gs_tune_cache_get")
    return rc.astuple(), float(ms.value)


def check_warp_noalloc_args(cam, device, rgb_dom, depth_dom, trans_dom, rgb_warp, depth_warp=None, hole=None):
    """Argument checks of warp_noalloc, before anything reaches the device: every
    tensor contiguous, on `device`, of the dtype and element count the C entry
    point reads or writes for a cam.height x cam.width frame (rgb 3*H*W float32,
    depth and transmittance H*W float32, hole H*W uint8). The C entry point
    takes plain pointers and cannot see a short buffer, so a mis-sized output
    would be written out of bounds. Raises ValueError."""
    npix = int(cam.width) * int(cam.height)
    spec = (("rgb_dom", rgb_dom, torch.float32, 3), ("depth_dom", depth_dom, torch.float32, 1),
            ("trans_dom", trans_dom, torch.float32, 1), ("rgb_warp", rgb_warp, torch.float32, 3),
            ("depth_warp", depth_warp, torch.float32, 1), ("hole", hole, torch.uint8, 1))
    for name, t, dtype, planes in spec:
        if t is None:
            if name in ("depth_warp", "hole"):
                continue
            raise ValueError(f"warp_noalloc: {name} is required")
        if not isinstance(t, torch.Tensor) or not t.is_contiguous():
            raise ValueError(f"warp_noalloc: {name} must be a contiguous tensor")
        if t.device != torch.device(device):
            raise ValueError(f"warp_noalloc: {name} is on {t.device}, expected {device}")
        if t.dtype != dtype:
            raise ValueError(f"warp_noalloc: {name} is {t.dtype}, expected {dtype}")
        if t.numel() != planes * npix:
            raise ValueError(f"warp_noalloc: {name} has {t.numel()} elements, expected {planes} x {cam.height} x "
                             f"{cam.width} = {planes * npix}")


def warp_noalloc(rgb_dom, depth_dom, trans_dom, pose_dom, pose_aff, cam, rgb_warp, depth_warp=None, hole=None,
                 stream=None):
    """Depth-tested forward warp of a dominant-eye render into the affiliated eye
    through gs_warp_noalloc, which allocates no device memory (for callers inside
    a host application that owns the GPU memory pool). All tensors are caller-
    owned CUDA tensors on the current device: rgb_dom (3, H, W), depth_dom and
    trans_dom (H, W) float32 in; rgb_warp (3, H, W) float32, optional depth_warp
    (H, W) float32 and hole (H, W) uint8 out (checked by check_warp_noalloc_args).
    Calls that overlap on the GPU share one static scratch array and race:
    serialise them."""
    if not isinstance(rgb_dom, torch.Tensor) or not rgb_dom.is_cuda:
        raise ValueError("warp_noalloc takes CUDA tensors")
    dev = torch.device("cuda", torch.cuda.current_device())
    check_warp_noalloc_args(cam, dev, rgb_dom, depth_dom, trans_dom, rgb_warp, depth_warp, hole)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    _check(lib().gs_warp_noalloc(_ptr(rgb_dom), _ptr(depth_dom), _ptr(trans_dom), C.byref(pose_struct(pose_dom)),
                                 C.byref(pose_struct(pose_aff)), C.byref(intr_struct(cam)), _ptr(rgb_warp),
                                 _ptr(depth_warp), _ptr(hole), C.c_void_p(st.cuda_stream)),
           "gs_warp_noalloc")
