"""FP64 CPU oracle (ctypes wrapper around liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline of bench.py. The CUDA path never imports it, and it imports nothing
from the CUDA path; only the seeded input generators (paper_2609_30741_gb300.synth)
feed both.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None


class OrScene(C.Structure):
    _fields_ = [("n", C.c_int), ("sh_degree", C.c_int), ("pos", C.c_void_p), ("quat", C.c_void_p),
                ("scale", C.c_void_p), ("opacity", C.c_void_p), ("sh", C.c_void_p), ("primitive", C.c_int)]


class OrPose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class OrCam(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("W", C.c_int), ("H", C.c_int)]


class OrParams(C.Structure):
    _fields_ = [("gap_thresh", C.c_int), ("margin", C.c_int), ("nsamples", C.c_int),
                ("enable_center", C.c_int), ("depth_mode", C.c_int), ("tile", C.c_int),
                ("dmin", C.c_double), ("dmax", C.c_double)]


class OrSplat(C.Structure):
    _fields_ = [("visible", C.c_int), ("pc", C.c_double * 3), ("M", C.c_double * 9),
                ("opacity", C.c_double), ("rc2", C.c_double), ("lp2", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("rgb", C.c_double * 3),
                ("key", C.c_float), ("box", C.c_double * 4), ("prim", C.c_int), ("conic", C.c_double * 3),
                ("su", C.c_double), ("sv", C.c_double), ("pscale", C.c_double)]


CLS_HOLE, CLS_GAP, CLS_CENTRE, CLS_STRIP, CLS_RENDER = 1, 2, 4, 8, 16


def lib():
    global _lib
    if _lib is None:
        path = _build()
        _lib = C.CDLL(path)
        _lib.or_eval.restype = C.c_double
        _lib.or_depth_range.restype = C.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _SceneRef:
    """Keeps the contiguous arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.arrays = [np.ascontiguousarray(a, dtype=np.float32) for a in
                       (scene.pos, scene.quat, scene.scale, scene.opacity, scene.sh)]
        self.s = OrScene(scene.n, scene.sh_degree, *[_p(a) for a in self.arrays], int(getattr(scene, "primitive", 0)))


def pose_struct(pose):
    return OrPose((C.c_double * 9)(*np.asarray(pose.R, np.float64).ravel()),
                  (C.c_double * 3)(*np.asarray(pose.t, np.float64).ravel()))


def cam_struct(cam):
    return OrCam(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)


def num_threads() -> int:
    return lib().or_num_threads()


def quat_to_rot(q):
    R = np.zeros(9)
    ok = lib().or_quat_to_rot(_p(np.ascontiguousarray(q, np.float32)), _p(R))
    return R.reshape(3, 3) if ok else None


def sh_basis(deg, d):
    Y = np.zeros(16)
    lib().or_sh_basis(C.c_int(deg), _p(np.ascontiguousarray(d, np.float64)), _p(Y))
    return Y[: (deg + 1) ** 2]


def prepare(scene, pose, cam):
    ref = _SceneRef(scene)
    out = (OrSplat * max(scene.n, 1))()
    lib().or_prepare(C.byref(ref.s), C.byref(pose_struct(pose)), C.byref(cam_struct(cam)), out)
    return out


def eval_pair(splat, cam, x, y):
    """(o * Ghat, depth, rho3, rho2) for one surfel and one pixel."""
    d, r3, r2 = C.c_double(), C.c_double(), C.c_double()
    oG = lib().or_eval(C.byref(splat), C.byref(cam_struct(cam)), C.c_double(x), C.c_double(y),
                       C.byref(d), C.byref(r3), C.byref(r2))
    return oG, d.value, r3.value, r2.value


def rho3_err(splat, cam, x, y, rho3, lam):
    """First-order bound on the float32 error of rho3 at pixel (x, y)."""
    lib().or_rho3_err.restype = C.c_double
    return lib().or_rho3_err(C.byref(splat), C.byref(cam_struct(cam)), C.c_double(x), C.c_double(y),
                             C.c_double(rho3), C.c_double(lam))


def render(scene, pose, cam, bg=(0.0, 0.0, 0.0), window=None, fp32_bound=False):
    """Full render of `window` = (x0, y0, w, h) (default: the whole image).
    Returns rgb [3,h,w], depth [h,w], trans [h,w], margin [h,w], pairs, and with
    fp32_bound=True also the per-pixel bound [h,w] on the error of a float32
    evaluation of the same sum; the margins then also account for the float32
    error of each surfel's rho3."""
    x0, y0, w, h = window if window is not None else (0, 0, cam.width, cam.height)
    rgb = np.zeros((3, h, w))
    dep = np.zeros((h, w))
    tr = np.zeros((h, w))
    mrg = np.zeros((h, w))
    pairs = C.c_int64()
    ref = _SceneRef(scene)
    bgv = np.asarray(bg, np.float64)
    bound = np.zeros((h, w)) if fp32_bound else None
    r = lib().or_render(C.byref(ref.s), C.byref(pose_struct(pose)), C.byref(cam_struct(cam)), _p(bgv),
                        x0, y0, w, h, _p(rgb), _p(dep), _p(tr), _p(mrg), C.byref(pairs), _p(bound))
    if r < 0:
        raise ValueError("oracle render: bad arguments")
    if fp32_bound:
        return rgb, dep, tr, mrg, pairs.value, bound
    return rgb, dep, tr, mrg, pairs.value


def render_tiles(scene, pose, cam, tile_mask, tile=16, bg=(0.0, 0.0, 0.0)):
    W, H = cam.width, cam.height
    rgb = np.zeros((3, H, W))
    dep = np.zeros((H, W))
    tr = np.ones((H, W))
    ref = _SceneRef(scene)
    mask = np.ascontiguousarray(tile_mask, np.uint8)
    lib().or_render_tiles(C.byref(ref.s), C.byref(pose_struct(pose)), C.byref(cam_struct(cam)),
                          _p(np.asarray(bg, np.float64)), tile, _p(mask), _p(rgb), _p(dep), _p(tr))
    return rgb, dep, tr


def tile_rect(bounds, W, H, tile=16):
    r = np.zeros(4, np.int32)
    b = np.ascontiguousarray(bounds, np.float32)
    cnt = lib().or_tile_rect(_p(b), W, H, tile, _p(r))
    return r, cnt


def depth_key(pose, p):
    """The oracle's depth-order key of a centre p (3 floats) for a pose."""
    lib().or_depth_key.restype = C.c_float
    pp = np.ascontiguousarray(p, np.float32)
    return float(lib().or_depth_key(C.byref(pose_struct(pose)), _p(pp)))


def sort_pairs(keys, vals):
    k = np.ascontiguousarray(keys, np.uint64).copy()
    v = np.ascontiguousarray(vals, np.uint32).copy()
    lib().or_sort_pairs(C.c_int64(k.size), _p(k), _p(v))
    return k, v


def warp(cam, src, dst, rgb, D, T):
    W, H = cam.width, cam.height
    n = W * H
    rgb = np.ascontiguousarray(rgb, np.float64)
    D = np.ascontiguousarray(D, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    tgt = np.zeros(n, np.int64)
    zkey = np.zeros(n, np.float32)
    tm = np.zeros(n)
    win = np.zeros(n, np.int64)
    zd = np.zeros(n, np.float32)
    out = np.zeros((3, H, W))
    hole = np.zeros((H, W), np.uint8)
    lib().or_warp(C.byref(cam_struct(cam)), C.byref(pose_struct(src)), C.byref(pose_struct(dst)),
                  _p(rgb), _p(D), _p(T), _p(tgt), _p(zkey), _p(tm), _p(win), _p(zd), _p(out), _p(hole))
    return dict(tgt=tgt, zkey=zkey, tmargin=tm, winner=win.reshape(H, W), zdst=zd.reshape(H, W),
                rgb=out, hole=hole)


def depth_range(D, T):
    D = np.ascontiguousarray(D, np.float64).ravel()
    T = np.ascontiguousarray(T, np.float64).ravel()
    lo, hi = C.c_double(), C.c_double()
    cnt = lib().or_depth_range(D.size, _p(D), _p(T), C.byref(lo), C.byref(hi))
    return lo.value, hi.value, cnt


def edge_roi(cam, src, dst, dmin, dmax, nsamples=32, m=32, tile=16):
    widths = np.zeros(4, np.int32)
    strips = np.zeros(16, np.int32)
    mrg = C.c_double()
    lib().or_edge_roi(C.byref(cam_struct(cam)), C.byref(pose_struct(src)), C.byref(pose_struct(dst)),
                      nsamples, C.c_double(dmin), C.c_double(dmax), m, tile, _p(widths), _p(strips),
                      C.byref(mrg))
    return widths, strips.reshape(4, 4), mrg.value


def strip_mask(strips, W, H):
    m = np.zeros((H, W), np.uint8)
    for x0, y0, x1, y1 in np.asarray(strips).reshape(-1, 4):
        m[y0:y1, x0:x1] = 1
    return m


def classify(hole, rgb, in_strip, gap_thresh=2, center_enabled=1):
    H, W = hole.shape
    hole = np.ascontiguousarray(hole, np.uint8)
    rgb = np.ascontiguousarray(rgb, np.float64)
    strip = np.ascontiguousarray(in_strip, np.uint8)
    cls = np.zeros((H, W), np.uint8)
    out = np.zeros((3, H, W))
    lib().or_classify(W, H, _p(hole), _p(rgb), _p(strip), gap_thresh, center_enabled, _p(cls), _p(out))
    return cls, out


def center_rois(cls, m=32, tile=16, cap=1 << 16):
    H, W = cls.shape
    cls = np.ascontiguousarray(cls, np.uint8)
    rects = np.zeros((cap, 4), np.int32)
    n = lib().or_center_rois(W, H, _p(cls), m, tile, _p(rects), cap)
    return rects[: min(n, cap)].copy(), n


def stereo(scene, dom, aff, cam, gap_thresh=2, margin=32, nsamples=32, enable_center=1,
           depth_mode=0, dmin=0.0, dmax=0.0, tile=16, bg=(0.0, 0.0, 0.0), rect_cap=1 << 16):
    W, H = cam.width, cam.height
    rgb_dom = np.zeros((3, H, W))
    dd = np.zeros((H, W))
    td = np.zeros((H, W))
    rgb_aff = np.zeros((3, H, W))
    cls = np.zeros((H, W), np.uint8)
    widths = np.zeros(4, np.int32)
    rects = np.zeros((rect_cap, 4), np.int32)
    nrects = C.c_int()
    ntx, nty = (W + tile - 1) // tile, (H + tile - 1) // tile
    tmask = np.zeros((nty, ntx), np.uint8)
    prm = OrParams(gap_thresh, margin, nsamples, enable_center, depth_mode, tile, dmin, dmax)
    ref = _SceneRef(scene)
    r = lib().or_stereo(C.byref(ref.s), C.byref(pose_struct(dom)), C.byref(pose_struct(aff)),
                        C.byref(cam_struct(cam)), _p(np.asarray(bg, np.float64)), C.byref(prm),
                        _p(rgb_dom), _p(dd), _p(td), _p(rgb_aff), _p(cls), _p(widths), _p(rects),
                        rect_cap, C.byref(nrects), _p(tmask))
    if r != 0:
        raise ValueError("oracle stereo: bad arguments")
    return dict(rgb_dom=rgb_dom, depth_dom=dd, trans_dom=td, rgb_aff=rgb_aff, cls=cls,
                widths=widths, rects=rects[: min(nrects.value, rect_cap)].copy(),
                nrects=nrects.value, tile_mask=tmask)


def support_pairs(scene, pose, cam, tile=16, cap=1 << 26):
    """(surfel ids, tile ids) of every pair whose tile holds a pixel centre with
    alpha >= 1/255, surfels in index order, tiles ascending per surfel."""
    ref = _SceneRef(scene)
    ids = np.zeros(cap, np.uint32)
    tiles = np.zeros(cap, np.uint32)
    lib().or_support_pairs.restype = C.c_int64
    n = lib().or_support_pairs(C.byref(ref.s), C.byref(pose_struct(pose)), C.byref(cam_struct(cam)), tile,
                               C.c_int64(cap), _p(ids), _p(tiles))
    if n > cap:
        raise ValueError("support_pairs: capacity too small")
    return ids[:n].copy(), tiles[:n].copy()


def tile_test(rec12, k, x0, x1, y0, y1):
    r = np.ascontiguousarray(rec12, np.float32)
    return bool(lib().or_tile_test(_p(r), C.c_double(k), C.c_double(x0), C.c_double(x1), C.c_double(y0),
                                   C.c_double(y1)))
