"""Seeded synthetic scenes and camera poses shaped like the paper's workloads.

This module only draws inputs: surfel attributes and eye poses in the layout the
C-ABI takes. It holds none of the method's arithmetic (no projection, no SH
evaluation, no blending), so both the CUDA path and the FP64 oracle can be fed
from it without sharing any computation.

Layouts (all float32, C-contiguous):
  pos      [n, 4]   surfel centre p_k (x, y, z) + an unused pad lane   (Sec. 3.3)
  quat     [n, 4]   rotation quaternion (w, x, y, z), unit norm         (Sec. 3.3)
  scale    [n, 2]   in-plane scales (s_u, s_v)                          (Eq. 1)
  opacity  [n]      opacity in (0, 1)
  sh       [n, (deg+1)^2, 3] real spherical-harmonic colour coefficients

Poses are camera-to-world (R, t) in float64 with OpenCV axes (x right, y down,
z forward), i.e. P_world = R X_cam + t as in Eq. 4. The dominant eye and the
affiliated eye share their orientation and differ by a small offset along the
camera x axis (Sec. 4.2).

The scene recipes follow the workload descriptions (scene sizes, shapes and
value distributions); the datasets the paper used (DTU, Tanks and Temples,
MipNeRF-360) are not available, and these synthetic scenes stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASELINE_M = 0.064  # interocular offset between the two eyes, metres


@dataclass
class Scene:
    pos: np.ndarray
    quat: np.ndarray
    scale: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    sh_degree: int
    primitive: int = 0  # 0: 2D surfels, scale [n][2]; 1: 3D ellipsoids, scale [n][4] (sx, sy, sz, 0)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.pos[idx].copy(), self.quat[idx].copy(), self.scale[idx].copy(),
                     self.opacity[idx].copy(), self.sh[idx].copy(), self.sh_degree, self.primitive)

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.pos, self.quat, self.scale, self.opacity, self.sh))


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclass
class Pose:
    R: np.ndarray  # [3, 3] float64 camera-to-world rotation
    t: np.ndarray  # [3] float64 camera centre in world coordinates


def centred_camera(width: int, height: int, f: float) -> Camera:
    """Pinhole camera with its principal point at the image centre; pixel centres
    sit at integer coordinates 0..W-1, so the centre is (W-1)/2, (H-1)/2."""
    return Camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height)


def _random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _lognormal_scales(rng, n, mu=math.log(0.02), sigma=0.5):
    return np.exp(rng.normal(mu, sigma, size=(n, 2))).astype(np.float32)


def _sh_from_uniform_rgb(rng, n):
    """Degree-0 colour coefficients whose band-0 colour 0.5 + Y_00 c is uniform in
    [0, 1]; Y_00 = 1/(2 sqrt(pi)) makes that c uniform in [-sqrt(pi), sqrt(pi)]."""
    lim = math.sqrt(math.pi)
    return rng.uniform(-lim, lim, size=(n, 1, 3)).astype(np.float32)


def _pack(pos3, quat, scale, opacity, sh, deg) -> Scene:
    n = pos3.shape[0]
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = pos3
    return Scene(np.ascontiguousarray(pos), np.ascontiguousarray(quat, dtype=np.float32),
                 np.ascontiguousarray(scale, dtype=np.float32),
                 np.ascontiguousarray(opacity, dtype=np.float32),
                 np.ascontiguousarray(sh, dtype=np.float32), deg)


def _uniform_ball(rng, n, radius, centre):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0, 1, n) ** (1.0 / 3.0)
    return d * r[:, None] + np.asarray(centre)[None, :]


def scene_slab_ball(seed: int, n_bg: int = 16000, n_fg: int = 4000, sh_degree: int = 0) -> Scene:
    """Small scene: a background slab of surfels (x in [-2,2], y in [-1.5,1.5],
    z in [3,4] m) and a foreground ball (radius 0.5 m at z = 1.5 m) that creates
    disocclusions. SH degree 0, RGB uniform in [0,1], opacity U(0.3, 0.99),
    log-normal scales (mu = ln 0.02, sigma = 0.5), Gaussian-random rotations.
    With sh_degree > 0 the higher bands get N(0, 0.2) coefficients (as in the
    object scene) on top of the same DC colour."""
    rng = np.random.default_rng(seed)
    bg = np.stack([rng.uniform(-2, 2, n_bg), rng.uniform(-1.5, 1.5, n_bg),
                   rng.uniform(3, 4, n_bg)], axis=1)
    fg = _uniform_ball(rng, n_fg, 0.5, (0.0, 0.0, 1.5))
    pos = np.concatenate([bg, fg], 0)
    n = pos.shape[0]
    quat = _random_quats(rng, n)
    scale = _lognormal_scales(rng, n)
    opacity = rng.uniform(0.3, 0.99, n)
    sh = _sh_from_uniform_rgb(rng, n)
    if sh_degree > 0:
        K = (sh_degree + 1) ** 2
        sh = np.concatenate([sh.reshape(n, 1, 3), rng.normal(0.0, 0.2, (n, K - 1, 3))], 1)
    return _pack(pos, quat, scale, opacity, sh, sh_degree)


def _plane_quats(rng, n):
    """Quaternions whose surfel normal t_w points along +y (a ground plane with y
    down), with a uniformly random in-plane rotation: q = q_x(-90 deg) * q_z(phi)."""
    phi = rng.uniform(0, 2 * math.pi, n)
    a = math.cos(-math.pi / 4), math.sin(-math.pi / 4)  # half-angle of -90 deg about x
    cz, sz = np.cos(phi / 2), np.sin(phi / 2)
    # Hamilton product (a0, a1, 0, 0) * (cz, 0, 0, sz)
    w = a[0] * cz
    x = a[1] * cz
    y = -a[1] * sz
    z = a[0] * sz
    return np.stack([w, x, y, z], 1).astype(np.float32)


def scene_object_ground(seed: int, n: int = 500_000, sh_degree: int = 3,
                        ground_frac: float = 0.1) -> Scene:
    """Object-centric scene: (1 - ground_frac) of the surfels in an isotropic
    Gaussian cluster (sigma 0.3 m) centred at (0, 0, 2) m plus ground_frac on a
    ground plane y = +0.6 m (x in [-2,2], z in [0.5,4]) with normals along +y.
    SH coefficients N(0, 0.2) up to sh_degree."""
    rng = np.random.default_rng(seed)
    n_g = int(round(n * ground_frac))
    n_c = n - n_g
    cl = rng.normal(0.0, 0.3, (n_c, 3)) + np.array([0.0, 0.0, 2.0])
    gr = np.stack([rng.uniform(-2, 2, n_g), np.full(n_g, 0.6), rng.uniform(0.5, 4.0, n_g)], 1)
    pos = np.concatenate([cl, gr], 0)
    quat = np.concatenate([_random_quats(rng, n_c), _plane_quats(rng, n_g)], 0)
    scale = _lognormal_scales(rng, n)
    opacity = rng.uniform(0.3, 0.99, n)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.2, (n, K, 3))
    return _pack(pos, quat, scale, opacity, sh, sh_degree)


def scene_unbounded(seed: int, n: int = 1_500_000, sh_degree: int = 3,
                    centre_frac: float = 0.6) -> Scene:
    """Unbounded-scene shape: centre_frac of the surfels uniform in a 1 m ball at
    the origin (log-normal scales as above) and the rest on a spherical shell with
    radius uniform in [10, 30] m and log-uniform scales in [0.03, 0.3] m."""
    rng = np.random.default_rng(seed)
    n_c = int(round(n * centre_frac))
    n_s = n - n_c
    cl = _uniform_ball(rng, n_c, 1.0, (0.0, 0.0, 0.0))
    d = rng.standard_normal((n_s, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sh_pos = d * rng.uniform(10, 30, n_s)[:, None]
    pos = np.concatenate([cl, sh_pos], 0)
    quat = _random_quats(rng, n)
    scale = np.concatenate([_lognormal_scales(rng, n_c),
                            np.exp(rng.uniform(math.log(0.03), math.log(0.3), (n_s, 2)))], 0)
    opacity = rng.uniform(0.3, 0.99, n)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.2, (n, K, 3))
    return _pack(pos, quat, scale, opacity, sh, sh_degree)


# ----------------------------------------------------------------------------- poses

def look_at(eye, target) -> Pose:
    """Camera-to-world pose at `eye` looking at `target`, world y pointing down
    (OpenCV axes: columns of R are camera x (right), y (down), z (forward))."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return Pose(np.stack([x, y, z], 1), eye.copy())


def eye_pair(dominant: Pose, baseline: float = BASELINE_M):
    """(dominant, affiliated): the affiliated eye keeps the orientation and sits
    `baseline` metres along the dominant camera's +x axis (Sec. 4.2)."""
    aff = Pose(dominant.R.copy(), dominant.t + baseline * dominant.R[:, 0])
    return dominant, aff


def identity_pose() -> Pose:
    return Pose(np.eye(3), np.zeros(3))


def arc_poses(n: int = 8, centre=(0.0, 0.0, 2.0), radius: float = 2.0,
              arc_deg: float = 30.0):
    """n head poses spread evenly over a horizontal arc of arc_deg degrees around
    `centre` at `radius`, each looking at the centre; yaw 0 puts the eye at
    centre - radius * z."""
    c = np.asarray(centre, np.float64)
    out = []
    for k in range(n):
        yaw = math.radians(-arc_deg / 2 + arc_deg * k / max(n - 1, 1))
        eye = c + radius * np.array([math.sin(yaw), 0.0, -math.cos(yaw)])
        out.append(look_at(eye, c))
    return out


def yaw_trajectory(n_frames: int = 120, rate_deg_s: float = 60.0, hz: float = 90.0,
                   radius: float = 3.0, centre=(0.0, 0.0, 0.0)):
    """Head-pose trajectory orbiting `centre` at `radius` with a constant yaw rate,
    sampled at `hz`, each pose looking at the centre."""
    c = np.asarray(centre, np.float64)
    out = []
    for k in range(n_frames):
        yaw = math.radians(rate_deg_s * k / hz)
        eye = c + radius * np.array([math.sin(yaw), 0.0, -math.cos(yaw)])
        out.append(look_at(eye, c))
    return out


# ----------------------------------------------------------------------------- workloads

def workload_small(seed: int = 1100):
    """20k-surfel slab + ball scene, 256x192 pinhole (f = 300), dominant eye at
    the origin looking +z, affiliated eye 0.064 m along +x."""
    cam = centred_camera(256, 192, 300.0)
    dom, aff = eye_pair(identity_pose())
    return scene_slab_ball(seed), cam, dom, aff


def workload_object(seed: int = 1200, n: int = 500_000, pose_index: int = 0,
                    width: int = 1600, height: int = 1200, f: float = 1600.0):
    """500k-surfel object + ground scene (SH degree 3), 1600x1200 (f = 1600),
    head pose `pose_index` of 8 on a 30 degree arc, 0.064 m baseline."""
    cam = centred_camera(width, height, f)
    dom, aff = eye_pair(arc_poses()[pose_index])
    return scene_object_ground(seed, n), cam, dom, aff


def to_ellipsoids(scene: Scene, thickness: float = 0.1) -> Scene:
    """The same primitives as 3D Gaussians (the 3DGS backbone): tangent scales
    kept, a third axis along the surfel normal of `thickness` times the smaller
    tangent scale."""
    s = np.asarray(scene.scale, np.float32)
    sz = thickness * np.minimum(s[:, 0], s[:, 1])
    scale = np.stack([s[:, 0], s[:, 1], sz, np.zeros_like(sz)], 1).astype(np.float32)
    return Scene(scene.pos.copy(), scene.quat.copy(), scale, scene.opacity.copy(), scene.sh.copy(),
                 scene.sh_degree, 1)


def workload_batched(seed: int = 1500, scale: float = 1.0):
    """Four scenes of uneven size, each with four head poses (16 stereo frames),
    SH degree 3, 0.064 m baseline; per scene (scene, camera, [4 pose pairs]):
      200k slab + ball (small-scene distribution), 1280x720, f = 1500 (the small
          camera's field of view), the head 0.1 m around the origin looking +z;
      500k object + ground, 1600x1200, f = 1600, poses 0, 2, 5, 7 of the arc;
      1.2M object + ground, 1920x1080, f = 1920, poses 1, 3, 4, 6 of the arc;
      3M unbounded, 2048x1536, f = 1506 (the 2448-pixel, f = 1800 field of
          view), orbiting at 3 m with yaw 0, 10, 20, 30 degrees.
    `scale` shrinks every surfel count (tests)."""
    n = lambda k: max(int(round(k * scale)), 1000)
    fwd = [look_at((x, 0.0, 0.0), (0.0, 0.0, 3.5)) for x in (-0.1, -0.033, 0.033, 0.1)]
    arc = arc_poses()
    orbit = [look_at(3.0 * np.array([math.sin(math.radians(y)), 0.0, -math.cos(math.radians(y))]), (0.0, 0.0, 0.0))
             for y in (0.0, 10.0, 20.0, 30.0)]
    return [
        (scene_slab_ball(seed, n(160_000), n(40_000), sh_degree=3), centred_camera(1280, 720, 1500.0),
         [eye_pair(p) for p in fwd]),
        (scene_object_ground(seed + 1, n(500_000)), centred_camera(1600, 1200, 1600.0),
         [eye_pair(arc[k]) for k in (0, 2, 5, 7)]),
        (scene_object_ground(seed + 2, n(1_200_000)), centred_camera(1920, 1080, 1920.0),
         [eye_pair(arc[k]) for k in (1, 3, 4, 6)]),
        (scene_unbounded(seed + 3, n(3_000_000)), centred_camera(2048, 1536, 1506.0),
         [eye_pair(p) for p in orbit]),
    ]


def random_scene(seed: int, n: int, sh_degree: int = 0, z_range=(1.0, 4.0),
                 xy_half=(1.0, 0.75), scale_mu=math.log(0.05), scale_sigma=0.5,
                 opacity_range=(0.3, 0.99)) -> Scene:
    """Generic small scene for tests: centres uniform in a box in front of an
    identity camera, random rotations and colours."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(z_range[0], z_range[1], n)
    pos = np.stack([rng.uniform(-xy_half[0], xy_half[0], n) * z / 2,
                    rng.uniform(-xy_half[1], xy_half[1], n) * z / 2, z], 1)
    quat = _random_quats(rng, n)
    scale = np.exp(rng.normal(scale_mu, scale_sigma, (n, 2))).astype(np.float32)
    opacity = rng.uniform(opacity_range[0], opacity_range[1], n)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.5, (n, K, 3))
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    return _pack(pos, quat, scale, opacity, sh, sh_degree)


def fronto_parallel_plane(z: float, half_w: float, half_h: float, spacing: float,
                          s: float, opacity: float = 0.99, rgb_coeff=(0.0, 0.0, 0.0),
                          x_offset: float = 0.0) -> Scene:
    """A grid of identity-rotation surfels (normal along the optical axis) at depth
    z, spacing `spacing`, scales (s, s), constant opacity and degree-0 colour
    coefficients `rgb_coeff` (the same for every surfel)."""
    xs = np.arange(-half_w, half_w + 1e-9, spacing) + x_offset
    ys = np.arange(-half_h, half_h + 1e-9, spacing)
    X, Y = np.meshgrid(xs, ys)
    n = X.size
    pos = np.stack([X.ravel(), Y.ravel(), np.full(n, z)], 1)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    scale = np.full((n, 2), s, np.float32)
    op = np.full(n, opacity, np.float32)
    sh = np.tile(np.asarray(rgb_coeff, np.float32).reshape(1, 1, 3), (n, 1, 1))
    return _pack(pos, quat, scale, op, sh, 0)


def concat(*scenes: Scene) -> Scene:
    deg = max(s.sh_degree for s in scenes)
    K = (deg + 1) ** 2
    shs = []
    for s in scenes:
        pad = np.zeros((s.n, K, 3), np.float32)
        pad[:, : s.sh.shape[1], :] = s.sh
        shs.append(pad)
    return Scene(np.concatenate([s.pos for s in scenes]), np.concatenate([s.quat for s in scenes]),
                 np.concatenate([s.scale for s in scenes]), np.concatenate([s.opacity for s in scenes]),
                 np.concatenate(shs), deg)
