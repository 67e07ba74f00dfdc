"""Pins of the FP64 oracle to things other than itself: closed forms derived from
the paper's equations, library routines (scipy, numpy), an independent
ray-plane formulation on tiny scenes, invariants, and special cases.

CPU only (no GPU marker)."""
import json
import math
import os

import numpy as np
import pytest

from paper_2609_30741_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


# ----------------------------------------------------------------------------- independent helpers

def rot_from_quat_scipy(q):
    from scipy.spatial.transform import Rotation
    w, x, y, z = [float(v) for v in q]
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def brute_force_render(scene, pose, cam, bg=(0, 0, 0)):
    """Independent restatement: ray-plane intersection through the surfel normal
    (lambda = n.p / n.r), local coordinates by projecting onto the tangent axes,
    numpy loops over pixels, scipy rotations. Same blending rule."""
    W, H = cam.width, cam.height
    R, t = pose.R, pose.t
    items = []
    for i in range(scene.n):
        q = scene.quat[i]
        if not np.any(q):
            continue
        o = float(scene.opacity[i])
        if 255 * o < 1:
            continue
        Rq = rot_from_quat_scipy(q)
        p = scene.pos[i, :3].astype(np.float64)
        pc = R.T @ (p - t)
        tu, tv = R.T @ Rq[:, 0], R.T @ Rq[:, 1]
        n = np.cross(tu, tv)
        su, sv = float(scene.scale[i, 0]), float(scene.scale[i, 1])
        if pc[2] <= 0.2:
            continue
        rc = math.sqrt(2 * math.log(255 * o))
        if any((pc + a * su * tu + b * sv * tv)[2] <= 0.2 for a in (-rc, rc) for b in (-rc, rc)):
            continue
        d = (p - t) / np.linalg.norm(p - t)
        from scipy.special import sph_harm_y  # noqa: F401  (only to fail early if missing)
        Y = real_sh_scipy(scene.sh_degree, d)
        rgb = np.maximum(0.0, 0.5 + Y @ scene.sh[i].astype(np.float64))
        c = (cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy)
        items.append((np.float32(pc[2]), i, pc, tu, tv, n, su, sv, o, rgb, c))
    items.sort(key=lambda it: (it[0], it[1]))
    out = np.zeros((3, H, W))
    dep = np.zeros((H, W))
    tr = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            r = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
            T, C, D = 1.0, np.zeros(3), 0.0
            for (_, _, pc, tu, tv, n, su, sv, o, rgb, c) in items:
                nr = n @ r
                rho3, lam = math.inf, 0.0
                if nr != 0:
                    lam = (n @ pc) / nr
                    if lam > 0:
                        P = lam * r
                        u = (P - pc) @ tu / (su * (tu @ tu))
                        v = (P - pc) @ tv / (sv * (tv @ tv))
                        rho3 = u * u + v * v
                rho2 = 2 * ((x - c[0]) ** 2 + (y - c[1]) ** 2)
                G = math.exp(-0.5 * min(rho3, rho2))
                a = min(0.99, o * G)
                if a < 1 / 255:
                    continue
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                dd = lam if rho3 <= rho2 else pc[2]
                C += a * T * rgb
                D += a * T * dd
                T = Tn
            out[:, y, x] = C + T * np.asarray(bg)
            dep[y, x] = D
            tr[y, x] = T
    return out, dep, tr


def real_sh_scipy(deg, d):
    """Real SH from scipy's complex Y_l^m (sph_harm_y(l, m, theta, phi), which
    carries the Condon-Shortley phase): m > 0 -> sqrt(2) Re Y_l^m, m < 0 ->
    sqrt(2) Im Y_l^|m|, m = 0 -> Y_l^0, ordered m = -l..l (the ordering the colour
    coefficients use). Keeping the phase gives the 3DGS sign convention
    (-c y, c z, -c x for band 1)."""
    from scipy.special import sph_harm_y
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    out = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            Ylm = complex(sph_harm_y(l, abs(m), theta, phi))
            if m > 0:
                out.append(math.sqrt(2) * Ylm.real)
            elif m < 0:
                out.append(math.sqrt(2) * Ylm.imag)
            else:
                out.append(Ylm.real)
    return np.array(out)


# ----------------------------------------------------------------------------- geometry pins

def test_quaternion_rotation_matches_scipy(orc):
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.standard_normal(4).astype(np.float32)
        R = orc.quat_to_rot(q)
        np.testing.assert_allclose(R, rot_from_quat_scipy(q), atol=1e-12)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-12
    assert orc.quat_to_rot(np.zeros(4, np.float32)) is None


def test_sh_basis_matches_scipy_real_harmonics(orc):
    """The basis is scipy's complex SH turned real (Condon-Shortley phase), for
    every band up to 3, at random directions."""
    rng = np.random.default_rng(1)
    for _ in range(40):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        np.testing.assert_allclose(orc.sh_basis(3, d), real_sh_scipy(3, d), atol=1e-12)


def test_sh_basis_orthonormal_on_sphere(orc):
    """Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly."""
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 16
    G = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = orc.sh_basis(3, np.array([st * math.cos(ph), st * math.sin(ph), ct]))
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def f32(v):
    """The value the float32 scene arrays actually hold."""
    return float(np.float32(v))


def _one_surfel(pos, quat, s, o, rgb_coeff):
    return synth.Scene(np.array([[*pos, 0]], np.float32), np.array([quat], np.float32),
                       np.array([s], np.float32), np.array([o], np.float32),
                       np.array([[rgb_coeff]], np.float32), 0)


def test_single_surfel_closed_form(orc):
    """Fronto-parallel surfel at (0, 0, z), identity rotation: the ray of pixel
    (x, y) meets the plane at u = (x - cx) z / (fx s_u), v = (y - cy) z / (fy s_v)
    (Eq. 1-3), so the pixel value is min(0.99, o G) c with G = exp(-(u^2+v^2)/2)
    (Eq. 2) wherever the 3D term dominates the low-pass term."""
    cam = synth.centred_camera(48, 40, 300.0)
    z, su, sv, o = 2.0, f32(0.03), f32(0.05), f32(0.8)
    coeff = f32(1.0 / (0.5 / math.sqrt(math.pi)))  # colour 0.5 + Y00 * coeff ~ 1.5
    sc = _one_surfel((0, 0, z), (1, 0, 0, 0), (su, sv), o, (coeff, 0.0, -coeff))
    rgb, dep, tr, _, _ = orc.render(sc, synth.identity_pose(), cam)
    col = np.array([0.5 + 0.5 / math.sqrt(math.pi) * c for c in (coeff, 0.0, -coeff)])
    col = np.maximum(col, 0)
    for y in range(cam.height):
        for x in range(cam.width):
            u = (x - cam.cx) * z / (cam.fx * su)
            v = (y - cam.cy) * z / (cam.fy * sv)
            rho3 = u * u + v * v
            rho2 = 2 * ((x - cam.cx) ** 2 + (y - cam.cy) ** 2)
            a = min(0.99, o * math.exp(-0.5 * min(rho3, rho2)))
            if a < 1 / 255:
                a = 0.0
            np.testing.assert_allclose(rgb[:, y, x], a * col, atol=1e-12)
            np.testing.assert_allclose(tr[y, x], 1 - a, atol=1e-12)
            np.testing.assert_allclose(dep[y, x], a * z, atol=1e-12)


def test_low_pass_term_near_tiny_surfel(orc):
    """A surfel far below a pixel in size: near its projected centre c the low-pass
    term exp(-|x - c|^2) dominates and the contribution's depth is the centre depth."""
    cam = synth.centred_camera(9, 9, 300.0)
    sc = _one_surfel((0, 0, 2.0), (1, 0, 0, 0), (1e-4, 1e-4), 0.9, (0.0, 0.0, 0.0))
    rgb, dep, tr, _, _ = orc.render(sc, synth.identity_pose(), cam)
    for (x, y) in [(4, 4), (5, 4), (4, 5), (5, 5)]:
        d2 = (x - cam.cx) ** 2 + (y - cam.cy) ** 2
        a = min(0.99, f32(0.9) * math.exp(-d2))
        a = a if a >= 1 / 255 else 0.0
        np.testing.assert_allclose(1 - tr[y, x], a, atol=1e-12)
        np.testing.assert_allclose(dep[y, x], a * 2.0, atol=1e-12)
        np.testing.assert_allclose(rgb[:, y, x], a * 0.5, atol=1e-12)


def test_ray_splat_matches_ray_plane_formula(orc):
    """or_eval's 3x3 solve agrees with lambda = (n.p_c)/(n.r) and local coordinates
    from projecting onto the tangent axes, for random tilted surfels."""
    rng = np.random.default_rng(3)
    cam = synth.centred_camera(64, 48, 200.0)
    sc = synth.random_scene(5, 40, z_range=(1.0, 3.0), scale_mu=math.log(0.1))
    sp = orc.prepare(sc, synth.identity_pose(), cam)
    checked = 0
    for i in range(sc.n):
        s = sp[i]
        if not s.visible:
            continue
        Rq = rot_from_quat_scipy(sc.quat[i])
        pc = np.array(s.pc[:])
        tu, tv = Rq[:, 0], Rq[:, 1]
        n = np.cross(tu, tv)
        su, sv = float(sc.scale[i, 0]), float(sc.scale[i, 1])
        for _ in range(20):
            x, y = rng.uniform(0, 63), rng.uniform(0, 47)
            r = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
            lam = (n @ pc) / (n @ r)
            _, dep, rho3, rho2 = orc.eval_pair(s, cam, x, y)
            if lam <= 0:
                assert math.isinf(rho3)
                continue
            P = lam * r
            u, v = (P - pc) @ tu / su, (P - pc) @ tv / sv
            np.testing.assert_allclose(rho3, u * u + v * v, rtol=1e-9, atol=1e-9)
            if rho3 <= rho2:
                np.testing.assert_allclose(dep, lam, rtol=1e-12)
            checked += 1
    assert checked > 300


def test_brute_force_tiny_scenes(orc):
    """Up to 10 surfels: the oracle render equals an independent numpy brute force."""
    cam = synth.centred_camera(24, 18, 40.0)
    for seed in range(4):
        sc = synth.random_scene(seed, 3 + 2 * seed, sh_degree=seed % 4, z_range=(1.0, 3.0),
                                scale_mu=math.log(0.2), scale_sigma=0.4)
        pose = synth.identity_pose() if seed % 2 == 0 else synth.look_at((0.1, -0.05, -0.2), (0.0, 0.0, 2.0))
        rgb, dep, tr, _, _ = orc.render(sc, pose, cam, bg=(0.1, 0.2, 0.3))
        r2, d2, t2 = brute_force_render(sc, pose, cam, bg=(0.1, 0.2, 0.3))
        np.testing.assert_allclose(rgb, r2, atol=1e-10)
        np.testing.assert_allclose(dep, d2, atol=1e-10)
        np.testing.assert_allclose(tr, t2, atol=1e-12)


def test_weights_and_transmittance_sum_to_one(orc):
    """sum_i w_i + T_final = 1 (telescoping product of the blending rule): with
    every colour 1 and a black background, C + T = 1 at every pixel."""
    sc, cam, dom, _ = synth.workload_small()
    sc = sc.subset(np.arange(0, sc.n, 7))
    lim = math.sqrt(math.pi)
    sc.sh[:] = lim  # colour 0.5 + Y00 sqrt(pi) = 1
    rgb, dep, tr, _, _ = orc.render(sc, dom, cam, window=(64, 48, 96, 64))
    for ch in range(3):
        np.testing.assert_allclose(rgb[ch] + tr, 1.0, atol=1e-12)


def test_two_surfel_hand_case(orc):
    """Two fronto-parallel surfels over the centre pixel: C = a1 c1 + a2 (1-a1) c2,
    T = (1-a1)(1-a2), D = a1 z1 + a2 (1-a1) z2, independent of the input order."""
    cam = synth.centred_camera(5, 5, 100.0)
    k = f32(1.0 / (0.5 / math.sqrt(math.pi)))
    near = ((0, 0, 1.0), (1, 0, 0, 0), (0.5, 0.5), 0.6, (k, 0, 0))   # red ~1.5, 0.5, 0.5
    far = ((0, 0, 2.0), (1, 0, 0, 0), (0.5, 0.5), 0.7, (0, k, 0))    # 0.5, ~1.5, 0.5
    hi = 0.5 + 0.5 / math.sqrt(math.pi) * k
    for order in ((near, far), (far, near)):
        sc = synth.concat(*[_one_surfel(*o) for o in order])
        rgb, dep, tr, _, _ = orc.render(sc, synth.identity_pose(), cam)
        a1, a2 = f32(0.6), f32(0.7)
        c1, c2 = np.array([hi, 0.5, 0.5]), np.array([0.5, hi, 0.5])
        np.testing.assert_allclose(rgb[:, 2, 2], a1 * c1 + a2 * (1 - a1) * c2, atol=1e-12)
        np.testing.assert_allclose(tr[2, 2], (1 - a1) * (1 - a2), atol=1e-12)
        np.testing.assert_allclose(dep[2, 2], a1 * 1.0 + a2 * (1 - a1) * 2.0, atol=1e-12)


def test_termination_and_clamp_rules(orc):
    """Stacked opaque surfels: alpha clamps to 0.99; the loop stops before the
    contribution that would take T below 1e-4."""
    cam = synth.centred_camera(3, 3, 100.0)
    k = f32(1.0 / (0.5 / math.sqrt(math.pi)))
    hi = 0.5 + 0.5 / math.sqrt(math.pi) * k
    layers = [_one_surfel((0, 0, 1.0 + 0.1 * i), (1, 0, 0, 0), (1.0, 1.0), 0.999, (k, k, k))
              for i in range(4)]
    sc = synth.concat(*layers)
    rgb, dep, tr, _, _ = orc.render(sc, synth.identity_pose(), cam)
    # T: 1 -> 0.01 -> 1e-4 (>= 1e-4? 0.01 * 0.01 rounds to just above or below)
    T, C = 1.0, 0.0
    for _ in range(4):
        Tn = T * (1 - 0.99)
        if Tn < 1e-4:
            break
        C += 0.99 * T * hi
        T = Tn
    np.testing.assert_allclose(tr[1, 1], T, rtol=1e-12)
    np.testing.assert_allclose(rgb[0, 1, 1], C, rtol=1e-12)


def test_support_box_is_conservative(orc):
    """Every (pixel, surfel) pair with alpha >= 1/255 lies inside the surfel's box."""
    cam = synth.centred_camera(80, 60, 120.0)
    sc = synth.random_scene(11, 60, z_range=(0.8, 3.0), scale_mu=math.log(0.08))
    sp = orc.prepare(sc, synth.identity_pose(), cam)
    ys, xs = np.mgrid[0:60, 0:80]
    inside = 0
    for i in range(sc.n):
        s = sp[i]
        if not s.visible:
            continue
        for x, y in zip(xs.ravel(), ys.ravel()):
            oG = orc.eval_pair(s, cam, float(x), float(y))[0]
            if min(oG, 0.99) >= 1 / 255:
                assert s.box[0] <= x <= s.box[1] and s.box[2] <= y <= s.box[3]
                inside += 1
    assert inside > 1000


def test_tile_rect_hand_cases(orc):
    r, c = orc.tile_rect([0.2, 15.9, 3.0, 3.0], 64, 48)
    assert list(r) == [0, 0, 0, 0] and c == 1
    r, c = orc.tile_rect([15.5, 16.0, 0.0, 47.0], 64, 48)
    assert list(r) == [1, 0, 1, 2] and c == 3  # pixel 16 only, all rows
    r, c = orc.tile_rect([15.1, 15.9, 0.0, 5.0], 64, 48)
    assert c == 0  # no pixel centre inside
    r, c = orc.tile_rect([-100.0, 1000.0, -5.0, 1e9], 64, 48)
    assert list(r) == [0, 0, 3, 2] and c == 12
    r, c = orc.tile_rect([64.2, 70.0, 0.0, 5.0], 64, 48)
    assert c == 0


def test_sort_pairs_is_stable_sort(orc):
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 50, 5000).astype(np.uint64) << np.uint64(32)
    vals = np.arange(5000, dtype=np.uint32)
    k, v = orc.sort_pairs(keys, vals)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[order]) and np.array_equal(v, vals[order])


# ----------------------------------------------------------------------------- reprojection pins

def _const_depth(cam, z):
    H, W = cam.height, cam.width
    rgb = np.random.default_rng(0).uniform(0, 1, (3, H, W))
    return rgb, np.full((H, W), z), np.zeros((H, W))


def test_identity_pose_warp_is_identity(orc):
    sc, cam, dom, _ = synth.workload_small()
    rgb, D, T, _, _ = orc.render(sc.subset(np.arange(0, sc.n, 3)), dom, cam)
    w = orc.warp(cam, dom, dom, rgb, D, T)
    assert not w["hole"].any()
    np.testing.assert_array_equal(w["winner"].ravel(), np.arange(cam.width * cam.height))
    np.testing.assert_array_equal(w["rgb"], rgb)


@pytest.mark.parametrize("case", ["fronto_plane_shift", "fronto_plane_shift_alt"])
def test_fronto_parallel_plane_shifts_by_fb_over_z(orc, case):
    g = GOLD[case]
    cam = synth.centred_camera(256, 192, g["f"])
    dom, aff = synth.eye_pair(synth.identity_pose(), g["baseline"])
    rgb, D, T = _const_depth(cam, g["z"])
    w = orc.warp(cam, dom, aff, rgb, D, T)
    s = g["shift_px"]
    W = cam.width
    for y in (0, 77, 191):
        for x in range(W):
            if x <= W - 1 - s:
                assert w["winner"][y, x] == y * W + x + s
            else:
                assert w["hole"][y, x]
    assert w["hole"].sum() == s * cam.height
    assert np.min(w["tmargin"][w["tgt"] >= 0]) > 0.4  # targets sit on pixel centres


def test_fronto_plane_rendered_then_warped(orc):
    """The same shift through the renderer: a dense opaque fronto-parallel plane at
    z = 3.2 renders with depth proxy 3.2 and warps by exactly 6 px."""
    cam = synth.centred_camera(64, 48, 300.0)
    dom, aff = synth.eye_pair(synth.identity_pose(), 0.064)
    plane = synth.fronto_parallel_plane(3.2, 0.5, 0.4, 0.01, 0.012, opacity=0.99)
    rgb, D, T, _, _ = orc.render(plane, dom, cam)
    assert T.max() < 0.5  # every pixel is a valid source
    np.testing.assert_allclose(D / (1 - T), f32(3.2), rtol=1e-12)
    w = orc.warp(cam, dom, aff, rgb, D, T)
    assert np.array_equal(np.where(w["hole"].any(0))[0], np.arange(64 - 6, 64))


def test_edge_roi_closed_form(orc):
    g = GOLD["edge_roi_plane"]
    cam = synth.centred_camera(g["W"], g["H"], g["f"])
    dom, aff = synth.eye_pair(synth.identity_pose(), g["baseline"])
    widths, strips, mrg = orc.edge_roi(cam, dom, aff, g["z"], g["z"], nsamples=32, m=g["m"], tile=g["tile"])
    assert list(widths) == g["widths"]
    assert list(strips[1]) == g["right_strip"]
    assert strips[0][2] == strips[0][0] and strips[2][3] == strips[2][1] and strips[3][3] == strips[3][1]


def _np_transfer(cam, src, dst, x, y, d):
    r = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
    P = src.R @ (r * d) + src.t
    X = dst.R.T @ (P - dst.t)
    return cam.fx * X[0] / X[2] + cam.cx, cam.fy * X[1] / X[2] + cam.cy, X[2]


def test_edge_roi_general_pose_against_numpy(orc):
    """Eq. 6-8 re-derived in numpy for rotated and translated eye pairs."""
    cam = synth.centred_camera(200, 150, 180.0)
    rng = np.random.default_rng(7)
    for k in range(12):
        base = synth.look_at(rng.normal(0, 0.3, 3), (rng.normal(0, 0.3), rng.normal(0, 0.3), 3.0))
        other = synth.look_at(base.t + rng.normal(0, 0.08, 3),
                              base.t + base.R[:, 2] * 3 + rng.normal(0, 0.2, 3))
        dmin, dmax = rng.uniform(0.8, 2.0), rng.uniform(2.0, 6.0)
        N, m, tile = 17, 32, 16
        widths, strips, mrg = orc.edge_roi(cam, base, other, dmin, dmax, nsamples=N, m=m, tile=tile)
        W, H = cam.width, cam.height
        pts = []
        for e in range(4):
            for kk in range(N):
                L = W if e < 2 else H
                pos = int(math.floor(kk * (L - 1) / (N - 1) + 0.5))
                x, y = [(pos, 0), (pos, H - 1), (0, pos), (W - 1, pos)][e]
                for d in (dmin, dmax):
                    u, v, z = _np_transfer(cam, base, other, x, y, d)
                    if z > 0.2:
                        pts.append((math.floor(u + 0.5), math.floor(v + 0.5)))
        pts = np.array(pts)
        xmin, xmax, ymin, ymax = pts[:, 0].min(), pts[:, 0].max(), pts[:, 1].min(), pts[:, 1].max()
        cl = lambda v, a, b: min(max(v, a), b)  # noqa: E731
        exp = [cl(xmin + m, 0, W // 2) if xmin > 0 else 0,
               cl((W - 1) - xmax + m, 0, W // 2) if xmax < W - 1 else 0,
               cl(ymin + m, 0, H // 2) if ymin > 0 else 0,
               cl((H - 1) - ymax + m, 0, H // 2) if ymax < H - 1 else 0]
        assert list(widths) == exp, (k, widths, exp)
        assert mrg > 1e-6


def test_classify_hand_cases(orc):
    W, H = 12, 6
    hole = np.zeros((H, W), np.uint8)
    rgb = np.zeros((3, H, W))
    rgb[0] = np.arange(W)[None, :] * 1.0      # red ramps along x
    rgb[1] = np.arange(H)[:, None] * 10.0     # green ramps along y
    hole[2, 4:6] = 1                          # 2-px horizontal run, bounded -> gap (horizontal)
    hole[0:4, 9] = 1                          # vertical run touching the top, 1-px horizontal run -> gap (horizontal)
    hole[5, 0] = 1                            # corner pixel: horizontal run unbounded, vertical unbounded -> centre
    strip = np.zeros((H, W), np.uint8)
    cls, out = orc.classify(hole, rgb, strip, gap_thresh=2, center_enabled=1)
    assert cls[2, 4] & 2 and cls[2, 5] & 2
    np.testing.assert_allclose(out[0, 2, 4], 4.0)  # lerp between x=3 (3.0) and x=6 (6.0) at 1/3
    np.testing.assert_allclose(out[0, 2, 5], 5.0)
    np.testing.assert_allclose(out[1, 2, 4], 20.0)
    assert all(cls[y, 9] & 2 for y in range(4))
    np.testing.assert_allclose(out[0, 0:4, 9], 9.0)
    assert cls[5, 0] & 4 and not cls[5, 0] & 2
    # a 3-px run is not a gap unless the other axis is short
    hole2 = np.zeros((H, W), np.uint8)
    hole2[1:4, 3:6] = 1                       # 3x3 block -> centre holes
    cls2, _ = orc.classify(hole2, rgb, strip, gap_thresh=2, center_enabled=1)
    assert (cls2[1:4, 3:6] & 4).all()
    # centre off: row fill between the nearest valid pixels
    cls3, out3 = orc.classify(hole2, rgb, strip, gap_thresh=2, center_enabled=0)
    np.testing.assert_allclose(out3[0, 2, 3:6], [3.0, 4.0, 5.0])
    # pixels in a strip are left to re-render
    strip[1:4, 3:6] = 1
    cls4, _ = orc.classify(hole2, rgb, strip, gap_thresh=2, center_enabled=1)
    assert (cls4[1:4, 3:6] == 1 | 8).all()


def test_center_rois_match_scipy_labels(orc):
    from scipy import ndimage
    rng = np.random.default_rng(9)
    for k in range(6):
        W, H = 97 + 13 * k, 61 + 7 * k
        mask = (rng.uniform(0, 1, (H, W)) < 0.04 + 0.05 * k).astype(np.uint8)
        cls = (mask * 4).astype(np.uint8)
        m, tile = [0, 5, 32][k % 3], 16
        rects, n = orc.center_rois(cls, m=m, tile=tile)
        lab, nl = ndimage.label(mask, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
        assert n == nl
        first = ndimage.minimum(np.arange(W * H).reshape(H, W), lab, index=np.arange(1, nl + 1))
        order = np.argsort(first)
        objs = ndimage.find_objects(lab)
        exp = []
        for j in order:
            sy, sx = objs[j]
            x0, x1, y0, y1 = sx.start, sx.stop - 1, sy.start, sy.stop - 1
            tx0, ty0 = max(0, x0 - m) // tile, max(0, y0 - m) // tile
            tx1 = min((x1 + m) // tile, (W + tile - 1) // tile - 1)
            ty1 = min((y1 + m) // tile, (H + tile - 1) // tile - 1)
            exp.append([tx0 * tile, ty0 * tile, min((tx1 + 1) * tile, W), min((ty1 + 1) * tile, H)])
        assert np.array_equal(rects, np.array(exp, np.int32).reshape(-1, 4))


def _disocclusion_setup(z_front):
    cam = synth.centred_camera(256, 192, 300.0)
    dom, aff = synth.eye_pair(synth.identity_pose(), 0.064)
    H, W = cam.height, cam.width
    D = np.full((H, W), 3.2)
    D[60:130, 100:160] = z_front  # occluder covering dom pixels x in [100, 160), y in [60, 130)
    rgb = np.random.default_rng(0).uniform(0, 1, (3, H, W))
    return cam, dom, aff, rgb, D, np.zeros((H, W))


def test_disocclusion_band_becomes_centre_roi(orc):
    g = GOLD["disocclusion_width"]
    cam, dom, aff, rgb, D, T = _disocclusion_setup(g["z_front"])
    w = orc.warp(cam, dom, aff, rgb, D, T)
    # foreground right edge: dom x = 159 -> aff 159 - 12 = 147; background dom 160 -> 154
    band = w["hole"][60:130, :200]
    cols = np.where(band.all(0))[0]
    assert list(cols) == list(range(148, 148 + g["width_px"]))
    dmin, dmax, _ = orc.depth_range(D, T)
    widths, strips, _ = orc.edge_roi(cam, dom, aff, dmin, dmax)
    sm = orc.strip_mask(strips, cam.width, cam.height)
    cls, _ = orc.classify(w["hole"], w["rgb"], sm, gap_thresh=2, center_enabled=1)
    rects, n = orc.center_rois(cls)
    assert n == 1
    # bbox x [148, 153], y [60, 129] -> expand 32 -> [116, 185] x [28, 161] -> tiles
    assert list(rects[0]) == [112, 16, 192, 176]


def test_narrow_disocclusion_is_all_gaps(orc):
    g = GOLD["disocclusion_gap"]
    cam, dom, aff, rgb, D, T = _disocclusion_setup(g["z_front"])
    w = orc.warp(cam, dom, aff, rgb, D, T)
    band = w["hole"][60:130, :200]
    assert list(np.where(band.all(0))[0]) == [159 - 8 + 1, 159 - 8 + 2]
    sm = np.zeros_like(w["hole"])
    cls, out = orc.classify(w["hole"], w["rgb"], sm, gap_thresh=2, center_enabled=1)
    inner = cls[60:130, 152:154]
    # the right-edge field-of-view band is not a gap; nothing left of it is a centre hole
    assert (inner & 2).all() and not (cls[:, :200] & 4).any()


def test_stereo_identity_pose_gives_identity_image(orc):
    sc, cam, dom, _ = synth.workload_small()
    sc = sc.subset(np.arange(0, sc.n, 5))
    out = orc.stereo(sc, dom, dom, cam)
    assert list(out["widths"]) == [0, 0, 0, 0]
    assert out["nrects"] == 0 and not out["tile_mask"].any()
    np.testing.assert_array_equal(out["rgb_aff"], out["rgb_dom"])


def test_render_window_matches_full_frame(orc):
    sc, cam, dom, _ = synth.workload_small()
    sc = sc.subset(np.arange(0, sc.n, 9))
    full = orc.render(sc, dom, cam)
    win = orc.render(sc, dom, cam, window=(40, 30, 70, 50))
    np.testing.assert_array_equal(win[0], full[0][:, 30:80, 40:110])
    np.testing.assert_array_equal(win[1], full[1][30:80, 40:110])


def test_stereo_composes_its_stages(orc):
    """or_stereo = warp -> edge ROI -> classify -> centre ROIs -> full affiliated
    render on the ROI tiles over the reprojected image."""
    sc, cam, dom, aff = synth.workload_small()
    sc = sc.subset(np.arange(0, sc.n, 4))
    out = orc.stereo(sc, dom, aff, cam)
    rgb, D, T, _, _ = orc.render(sc, dom, cam)
    np.testing.assert_array_equal(out["rgb_dom"], rgb)
    w = orc.warp(cam, dom, aff, rgb, D, T)
    dmin, dmax, _ = orc.depth_range(D, T)
    widths, strips, _ = orc.edge_roi(cam, dom, aff, dmin, dmax)
    assert list(widths) == list(out["widths"])
    sm = orc.strip_mask(strips, cam.width, cam.height)
    cls, filled = orc.classify(w["hole"], w["rgb"], sm)
    rects, n = orc.center_rois(cls)
    assert n == out["nrects"] and np.array_equal(rects, out["rects"])
    tm = np.zeros_like(out["tile_mask"])
    for x0, y0, x1, y1 in list(strips) + list(rects):
        if x1 > x0 and y1 > y0:
            tm[y0 // 16:(y1 - 1) // 16 + 1, x0 // 16:(x1 - 1) // 16 + 1] = 1
    assert np.array_equal(tm, out["tile_mask"])
    full = orc.render(sc, aff, cam)[0]
    pix = np.kron(tm, np.ones((16, 16), np.uint8))[: cam.height, : cam.width].astype(bool)
    np.testing.assert_array_equal(out["rgb_aff"][:, pix], full[:, pix])
    np.testing.assert_array_equal(out["rgb_aff"][:, ~pix], filled[:, ~pix])
    assert np.array_equal(out["cls"] & 15, cls) and np.array_equal((out["cls"] & 16) > 0, pix)


def test_tile_test_matches_dense_sampling(orc):
    """The conic-rectangle test agrees with a dense sampling of the rectangle
    wherever the sampled minimum is clearly away from the boundary."""
    rng = np.random.default_rng(21)
    checked = 0
    for _ in range(300):
        rec = np.zeros(12, np.float32)
        rec[0:2] = rng.uniform(-20, 20, 2)
        th = rng.uniform(0, np.pi)
        su, sv = rng.uniform(2, 30, 2)
        # an ellipse map: p.xy = R(th) diag(1/su, 1/sv) d scaled, p.z ~ 1 + small tilt
        Rm = np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]])
        Mxy = np.diag([1 / su, 1 / sv]) @ Rm
        rec[4], rec[6] = Mxy[0, 0], Mxy[0, 1]
        rec[5], rec[7] = Mxy[1, 0], Mxy[1, 1]
        rec[8] = 1.0
        rec[9:11] = rng.uniform(-0.01, 0.01, 2)
        k = float(rng.uniform(1, 11))
        x0, y0 = rng.uniform(-60, 40, 2)
        x1, y1 = x0 + 15, y0 + 15
        xs, ys = np.meshgrid(np.linspace(x0, x1, 121), np.linspace(y0, y1, 121))
        dx, dy = xs - rec[0], ys - rec[1]
        px = dx * rec[4] + dy * rec[6]
        py = dx * rec[5] + dy * rec[7]
        pz = rec[8] + dx * rec[9] + dy * rec[10]
        rho = (px ** 2 + py ** 2) / pz ** 2
        rho = np.minimum(rho, 2 * (dx ** 2 + dy ** 2))
        mn = rho.min()
        if abs(mn - k) < 0.05 * k:
            continue
        assert orc.tile_test(rec, k, x0, x1, y0, y1) == (mn <= k)
        checked += 1
    assert checked > 200


# ----------------------------------------------------------------------------- 3D Gaussian (ellipsoid) backbone

def _one_ellipsoid(pos, quat, scales, o, rgb_coeff):
    return synth.Scene(np.array([[*pos, 1.0]], np.float32), np.array([quat], np.float32),
                       np.array([[*scales, 0.0]], np.float32), np.array([o], np.float32),
                       np.array([[[c] for c in rgb_coeff]], np.float32).reshape(1, 1, 3), 0, 1)


def test_ellipsoid_on_axis_closed_form(orc):
    """An ellipsoid centred on the optical axis, rotated by theta about it: the
    Jacobian's depth column vanishes there, so the screen covariance is
    (f/z)^2 R2 diag(sa^2, sb^2) R2^T + 0.3 I, whatever the third scale."""
    f, z, th = 300.0, 3.0, 0.6
    sa, sb, sc_, o = 0.02, 0.008, 0.05, 0.8
    cam = synth.Camera(f, f, 64.0, 48.0, 129, 97)
    q = (math.cos(th / 2), 0.0, 0.0, math.sin(th / 2))
    coeff = (0.4, -0.2, 0.9)
    scene = _one_ellipsoid((0.0, 0.0, z), q, (sa, sb, sc_), o, coeff)
    rgb, dep, tr, _, _ = orc.render(scene, synth.identity_pose(), cam)
    # the values the float32 scene arrays hold
    R2 = rot_from_quat_scipy(np.asarray(scene.quat[0], np.float64))[:2, :2]
    sa, sb, o, z = f32(sa), f32(sb), f32(o), f32(z)
    S = (f / z) ** 2 * R2 @ np.diag([sa * sa, sb * sb]) @ R2.T + 0.3 * np.eye(2)
    Si = np.linalg.inv(S)
    col = np.maximum(0.0, 0.5 + 0.5 * math.sqrt(1.0 / math.pi) * np.array([f32(c) for c in coeff]))
    for (x, y) in ((64, 48), (66, 47), (61, 52), (70, 44)):
        d = np.array([x - 64.0, y - 48.0])
        a = o * math.exp(-0.5 * d @ Si @ d)
        if a < 1.0 / 255:
            assert tr[y, x] == 1.0
            continue
        a = min(a, 0.99)
        np.testing.assert_allclose(rgb[:, y, x], a * col, rtol=1e-12, atol=1e-15)
        assert abs(tr[y, x] - (1 - a)) < 1e-14 and abs(dep[y, x] - a * z) < 1e-12


def test_ellipsoid_off_axis_matches_numeric_jacobian(orc):
    """Off the axis the screen covariance is J V J^T + 0.3 I with J the
    projection's Jacobian at the centre: compare with central differences of the
    pinhole projection itself."""
    f = 250.0
    cam = synth.Camera(f, f, 80.0, 60.0, 161, 121)
    pos = np.array([0.4, -0.3, 2.5])
    q = np.array([0.8, 0.3, -0.4, 0.33])
    q /= np.linalg.norm(q)
    s = np.array([0.03, 0.012, 0.02])
    o = 0.9
    scene = _one_ellipsoid(tuple(pos), tuple(q), tuple(s), o, (1.0, 1.0, 1.0))
    rgb, _, tr, _, _ = orc.render(scene, synth.identity_pose(), cam)
    Rq = rot_from_quat_scipy(np.asarray(scene.quat[0], np.float64))
    V = Rq @ np.diag(s.astype(np.float32).astype(np.float64) ** 2) @ Rq.T

    def proj(X):
        return np.array([f * X[0] / X[2] + cam.cx, f * X[1] / X[2] + cam.cy])
    h = 1e-6
    J = np.stack([(proj(pos.astype(np.float32).astype(np.float64) + h * e) -
                   proj(pos.astype(np.float32).astype(np.float64) - h * e)) / (2 * h) for e in np.eye(3)], 1)
    S = J @ V @ J.T + 0.3 * np.eye(2)
    c = proj(pos.astype(np.float32).astype(np.float64))
    Si = np.linalg.inv(S)
    o = f32(o)
    checked = 0
    for y in range(121):
        for x in range(161):
            d = np.array([x, y]) - c
            a = o * math.exp(-0.5 * d @ Si @ d)
            if a < 2.0 / 255:
                continue
            assert abs((1.0 - tr[y, x]) - min(a, 0.99)) < 1e-8, (x, y)
            checked += 1
    assert checked > 20


def test_ellipsoid_weights_and_transmittance_sum_to_one(orc):
    # white colour, black background: the image is the sum of the weights
    rng = np.random.default_rng(41)
    base = synth.random_scene(42, 60, sh_degree=0, z_range=(1.5, 3.0), scale_mu=math.log(0.05))
    base.sh[:] = (0.5 / (0.5 * math.sqrt(1.0 / math.pi)))  # 0.5 + Y00 c = 1
    scene = synth.to_ellipsoids(base, thickness=0.5)
    cam = synth.centred_camera(64, 48, 60.0)
    rgb, _, tr, _, _ = orc.render(scene, synth.identity_pose(), cam)
    np.testing.assert_allclose(rgb[0] + tr, 1.0, atol=1e-12)
    assert (tr < 0.999).mean() > 0.3


def _brute_support_pairs(orc, scene, pose, cam, tile):
    """Every (surfel, tile) pair found by evaluating each visible surfel at every
    pixel centre of the whole image (no box, no early exit): the pair is kept when
    some pixel of the tile has min(0.99, o G) >= 1/255 (the skip rule of Stage 1)."""
    sp = orc.prepare(scene, pose, cam)
    ntx = (cam.width + tile - 1) // tile
    pairs = []
    for i in range(scene.n):
        s = sp[i]
        if not s.visible:
            continue
        hit = set()
        for y in range(cam.height):
            for x in range(cam.width):
                oG = orc.eval_pair(s, cam, float(x), float(y))[0]
                if min(oG, 0.99) >= 1 / 255:
                    hit.add((y // tile) * ntx + x // tile)
        pairs += [(i, t) for t in sorted(hit)]
    return pairs


@pytest.mark.parametrize("tile", [8, 16])
def test_support_pairs_match_whole_image_sweep(orc, tile):
    """or_support_pairs (which sweeps only each surfel's support box) against a
    sweep of or_eval over every pixel of the image, on a ragged image (37 x 29:
    neither side a multiple of the tile) with surfels whose boxes cross the
    left, right, top and bottom borders and corners, and under a tilted pose."""
    cam = synth.centred_camera(37, 29, 40.0)
    base = synth.random_scene(21, 10, z_range=(1.0, 2.5), scale_mu=math.log(0.15), scale_sigma=0.4)
    # surfels centred on or beyond the borders (x, y in camera units at z = 1.5:
    # the half field of view is 18 px / 40 * 1.5 = 0.675 m across, 0.525 m down)
    edge = []
    for k, (px, py) in enumerate([(-0.68, 0.0), (0.70, 0.1), (0.0, -0.55), (0.1, 0.56), (-0.7, -0.55),
                                  (0.66, 0.52), (-0.75, 0.3), (0.2, 0.6)]):
        q = np.array([1.0, 0.3 * (k % 3), -0.2 * (k % 2), 0.1 * k])
        edge.append(_one_surfel((px, py, 1.5), q / np.linalg.norm(q), (0.12, 0.08), 0.9, (0.0, 0.0, 0.0)))
    # small surfels centred one to three pixels outside a border (or on a tile
    # boundary), whose support reaches only the first or last pixel row or column
    # of the tiles it touches
    z, f = 1.5, 40.0
    for k, (u, v) in enumerate([(-2.0, 14.0), (38.5, 9.0), (20.0, -1.6), (11.0, 30.2), (-1.5, -1.5),
                                (39.0, 30.5), (7.5, 5.0), (15.5, 23.5), (24.0, 7.6)]):
        s = 0.02 + 0.006 * (k % 3)
        edge.append(_one_surfel(((u - cam.cx) * z / f, (v - cam.cy) * z / f, z), (1, 0, 0, 0), (s, s), 0.95,
                                (0.0, 0.0, 0.0)))
    sc = synth.concat(base, *edge)
    for pose in (synth.identity_pose(), synth.look_at((0.05, -0.03, -0.1), (0.02, 0.01, 1.8))):
        ids, tiles = orc.support_pairs(sc, pose, cam, tile=tile)
        got = list(zip(ids.tolist(), tiles.tolist()))
        want = _brute_support_pairs(orc, sc, pose, cam, tile)
        assert got == want
        # the scene does reach every border, and the ragged last column and row
        ntx, nty = (37 + tile - 1) // tile, (29 + tile - 1) // tile
        hit_tiles = {t for _, t in want}
        assert any(t % ntx == ntx - 1 for t in hit_tiles) and any(t // ntx == nty - 1 for t in hit_tiles)
        assert any(t % ntx == 0 for t in hit_tiles) and any(t // ntx == 0 for t in hit_tiles)
        assert len(want) > 30


def _round_f32(x):
    """Exact round-to-nearest-even of a Fraction to float32."""
    from fractions import Fraction
    c = np.float32(float(x))
    best = c
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d, db = abs(Fraction(float(cand)) - x), abs(Fraction(float(best)) - x)
        if d < db or (d == db and int(np.float32(cand).view(np.uint32)) % 2 == 0):
            best = cand
    return np.float32(best)


def test_depth_key_is_the_float32_camera_depth(orc):
    """The depth-order key is z = r20 x + r21 y + r22 z + t2 evaluated in float32
    with one rounding per fused multiply-add, the rotation row and offset rounded
    to float32 from the FP64 pose: checked against an exact-arithmetic restatement
    (fractions), and against the FP64 depth within a few float32 ulps."""
    from fractions import Fraction as F
    rng = np.random.default_rng(44)
    for k in range(200):
        pose = synth.look_at(rng.normal(0, 2, 3), rng.normal(0, 1, 3) + np.array([0.0, 0.0, 3.0]))
        p = rng.normal(0, 2, 3).astype(np.float32)
        R, t = np.asarray(pose.R, np.float64), np.asarray(pose.t, np.float64)
        t2 = 0.0
        for j in range(3):
            t2 = float(F(-R[j, 2]) * F(t[j]) + F(t2))  # fma in float64: exact, then one rounding
        r = [np.float32(R[j, 2]) for j in range(3)]
        z = _round_f32(F(float(r[2])) * F(float(p[2])) + F(float(np.float32(t2))))
        z = _round_f32(F(float(r[1])) * F(float(p[1])) + F(float(z)))
        z = _round_f32(F(float(r[0])) * F(float(p[0])) + F(float(z)))
        key = orc.depth_key(pose, p)
        assert key == float(z), (k, key, float(z))
        z64 = float(R[:, 2] @ (p.astype(np.float64) - t))
        assert abs(key - z64) <= 8 * abs(float(np.spacing(np.float32(z64)))) + 1e-6


def test_fp32_bound_covers_a_float32_blend(orc):
    """The oracle's per-pixel float32 error bound against an actual float32
    evaluation of the same blend: a stack of fronto-parallel surfels centred on
    the optical axis (so G = 1 at the centre pixel and alpha = min(0.99, o)),
    with low and high opacities mixed so that the stop rule is reached only after
    many contributions; numpy float32 arithmetic for alpha, T and the colour sum
    must stay within the bound of the FP64 result, and the bound must not be
    vacuous."""
    cam = synth.centred_camera(3, 3, 100.0)
    k = f32(1.0 / (0.5 / math.sqrt(math.pi)))
    for seed, hi_share in ((1, 0.0), (2, 0.15), (3, 0.4)):
        rng = np.random.default_rng(seed)
        n = 400
        z = 1.0 + np.arange(n) * 0.01
        o = np.where(rng.random(n) < hi_share, rng.uniform(0.85, 0.98, n), rng.uniform(0.005, 0.05, n))
        col = rng.uniform(0.0, 1.0, (n, 3))
        sc = synth.concat(*[_one_surfel((0, 0, z[i]), (1, 0, 0, 0), (1.0, 1.0), o[i],
                                        tuple(k * (c - 0.5) for c in col[i])) for i in range(n)])
        rgb, _, tr, _, _, bound = orc.render(sc, synth.identity_pose(), cam, window=(1, 1, 1, 1), fp32_bound=True)
        # float32 restatement of the blend at this pixel (alpha = min(0.99, o), G = 1)
        T, C = np.float32(1.0), np.zeros(3, np.float32)
        cs = (0.5 + (0.5 / math.sqrt(math.pi)) * sc.sh[:, 0, :].astype(np.float64)).astype(np.float32)
        for i in range(n):
            a = min(np.float32(0.99), np.float32(sc.opacity[i]))
            if a < np.float32(1 / 255):
                continue
            Tn = np.float32(T * np.float32(np.float32(1.0) - a))
            if Tn < np.float32(1e-4):
                break
            C = (C + cs[i] * np.float32(a * T)).astype(np.float32)
            T = Tn
        err = np.abs(C.astype(np.float64) - rgb[:, 0, 0]).max()
        assert err <= bound[0, 0], (seed, err, bound[0, 0])
        assert bound[0, 0] < 1e-3


def _quat_from_rot(R):
    from scipy.spatial.transform import Rotation
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return (w, x, y, z)


def test_rho3_uncertainty_covers_an_independent_float32_solve(orc):
    """The oracle's first-order bound on the float32 error of rho3 (or_rho3_err:
    one unit roundoff on each input magnitude, amplified by the ray's inverse
    cosine to the surfel normal) against an independent float32 evaluation:
    the world-to-camera transform as R^T (P - t) and a pivoted LU solve
    (numpy float32) of [s_u t_u, s_v t_v, -r] (u, v, lambda) = -p_c. Surfels 2-30 m
    from a rotated camera, half of them within 0.2-3 degrees of edge-on to the
    ray through the sampled pixel. The uncertainty must cover the independent
    error on every pair and must not be vacuous on well-conditioned pairs."""
    rng = np.random.default_rng(77)
    cam = synth.centred_camera(2000, 2000, 1800.0)
    pose = synth.look_at((2.5, -0.4, -3.0), (0.3, 0.1, 4.0))
    R, t = pose.R, pose.t
    n = 400
    rows = []
    for i in range(n):
        d = rng.uniform(2.0, 30.0)
        dirc = np.array([rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), 1.0])
        pc = d * dirc / np.linalg.norm(dirc)
        view = pc / np.linalg.norm(pc)
        if i % 2 == 0:  # nearly edge-on: the normal almost perpendicular to the view ray
            a = rng.standard_normal(3)
            tu = a - (a @ view) * view
            tu /= np.linalg.norm(tu)
            nrm0 = np.cross(view, tu)
            th = math.radians(rng.uniform(0.2, 3.0))
            nrm = math.cos(th) * nrm0 + math.sin(th) * view
            tv = np.cross(nrm, tu)
            Rc = np.stack([tu, tv, nrm], 1)
        else:
            from scipy.spatial.transform import Rotation
            Rc = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        Rw = R @ Rc  # tangent frame in world coordinates
        pw = R @ pc + t
        su, sv = rng.uniform(0.01, 0.1, 2)
        o = rng.uniform(0.2, 0.95)
        sc = _one_surfel(tuple(pw), _quat_from_rot(Rw), (su, sv), o, (0.0, 0.0, 0.0))
        sp = orc.prepare(sc, pose, cam)[0]
        if not sp.visible:
            continue
        # a pixel inside the support: a local point of the disc, projected
        rc = math.sqrt(sp.rc2)
        uv = rng.uniform(-0.7, 0.7, 2) * rc
        M = np.array(sp.M).reshape(3, 3)
        P = M @ np.array([uv[0], uv[1], 1.0])
        if P[2] <= 0.2:
            continue
        x, y = cam.fx * P[0] / P[2] + cam.cx, cam.fy * P[1] / P[2] + cam.cy
        _, lam, rho3, rho2 = orc.eval_pair(sp, cam, x, y)
        if not np.isfinite(rho3) or rho3 > rho2:
            continue
        err_bound = orc.rho3_err(sp, cam, x, y, rho3, lam)
        # independent float32 evaluation
        q = sc.quat[0].astype(np.float32)
        Rq = np.array(rot_from_quat_scipy(q), np.float32)
        Rt32 = R.T.astype(np.float32)
        pc32 = Rt32 @ (sc.pos[0, :3].astype(np.float32) - t.astype(np.float32))
        m0 = np.float32(sc.scale[0, 0]) * (Rt32 @ Rq[:, 0])
        m1 = np.float32(sc.scale[0, 1]) * (Rt32 @ Rq[:, 1])
        r32 = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0], np.float32)
        A = np.stack([m0, m1, -r32], 1).astype(np.float32)
        sol = np.linalg.solve(A, (-pc32).astype(np.float32)).astype(np.float32)
        rho3_32 = float(sol[0] * sol[0] + sol[1] * sol[1])
        rows.append((i % 2 == 0, abs(rho3_32 - rho3), err_bound, rho3))
    rows = np.array(rows, dtype=np.float64)
    assert len(rows) > 300
    grazing, err, bnd, rho = rows[:, 0] > 0, rows[:, 1], rows[:, 2], rows[:, 3]
    assert np.all(err <= bnd), np.max(err / bnd)
    # not vacuous: typically within a hundred times the independent error, and
    # edge-on pairs get far larger bounds than the others
    assert np.median(err / bnd) > 0.01
    assert np.median(bnd[grazing] / rho[grazing]) > 5 * np.median(bnd[~grazing] / rho[~grazing])
