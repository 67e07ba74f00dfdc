/*
 * Oracle, tile coverage. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper renders with the 2DGS tile rasterizer on 16x16 tiles (Sec. 3.5).
 * Tiling does not change the image as long as every (pixel, surfel) pair with
 * alpha >= 1/255 (the blending rule, Sec. 3.1 Stage 1) is binned to the
 * pixel's tile. The oracle states that set directly:
 *   or_support_pairs - every (surfel, tile) such that some pixel centre of the
 *                      tile has alpha >= 1/255, by evaluating the surfel at
 *                      every pixel of its support box (FP64);
 *   or_tile_test     - whether the continuous rectangle [x0,x1]x[y0,y1] meets
 *                      the support {u^2 + v^2 <= k} u {|x - c|^2 <= k/2} of a
 *                      surfel given in the blend-record form the GPU stores
 *                      (FP64, by the roots of the conic along each edge), so
 *                      the GPU's per-tile decisions can be compared on shared
 *                      inputs.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int64_t or_support_pairs(const or_scene *sc, const or_pose *pose, const or_cam *cam, int tile, int64_t cap,
                         uint32_t *ids, uint32_t *tiles) {
  or_splat *sp = (or_splat *)malloc(sizeof(or_splat) * (size_t)(sc->n > 0 ? sc->n : 1));
  or_prepare(sc, pose, cam, sp);
  const int W = cam->W, H = cam->H, ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
  uint8_t *hit = (uint8_t *)calloc((size_t)ntx * nty, 1);
  int64_t cnt = 0;
  for (int i = 0; i < sc->n; ++i) {
    const or_splat *s = &sp[i];
    if (!s->visible) continue;
    const int x0 = s->box[0] <= 0 ? 0 : (int)ceil(s->box[0]), x1 = s->box[1] >= W - 1 ? W - 1 : (int)floor(s->box[1]);
    const int y0 = s->box[2] <= 0 ? 0 : (int)ceil(s->box[2]), y1 = s->box[3] >= H - 1 ? H - 1 : (int)floor(s->box[3]);
    if (x0 > x1 || y0 > y1) continue;
    memset(hit, 0, (size_t)ntx * nty);
    for (int y = y0; y <= y1; ++y) {
      for (int x = x0; x <= x1; ++x) {
        const int t = (y / tile) * ntx + x / tile;
        if (hit[t]) continue;
        const double oG = or_eval(s, cam, x, y, NULL, NULL, NULL);
        if ((oG < OR_ALPHA_MAX ? oG : OR_ALPHA_MAX) >= OR_ALPHA_MIN) hit[t] = 1;
      }
    }
    for (int t = 0; t < ntx * nty; ++t) {
      if (!hit[t]) continue;
      if (cnt < cap) { ids[cnt] = (uint32_t)i; tiles[cnt] = (uint32_t)t; }
      ++cnt;
    }
  }
  free(hit);
  free(sp);
  return cnt;
}

/* Q(t) = A t^2 + 2 B t + C <= 0 for some t in [lo, hi]? (A > 0 for the ellipse) */
static int quad_has_nonpos(double A, double B, double C, double lo, double hi) {
  if (A * lo * lo + 2 * B * lo + C <= 0.0 || A * hi * hi + 2 * B * hi + C <= 0.0) return 1;
  if (A == 0.0) return 0;
  const double disc = B * B - A * C;
  if (disc < 0.0) return 0;
  const double sq = sqrt(disc);
  const double r1 = (-B - sq) / A, r2 = (-B + sq) / A;
  const double a = r1 < r2 ? r1 : r2, b = r1 < r2 ? r2 : r1;
  if (A > 0.0) return !(b < lo || a > hi); /* non-positive between the roots */
  return a >= lo || b <= hi;               /* concave: non-positive outside */
}

int or_tile_test(const float rec[12], double k, double x0, double x1, double y0, double y1) {
  /* rec: c.x, c.y, log2 o, z_c | V1, -V0, -U1, U0 | Az, Bz, Cz, dz_u */
  const double cx = rec[0], cy = rec[1];
  const double ax = rec[4], ay = rec[5], az = rec[9];
  const double bx = rec[6], by = rec[7], bz = rec[10];
  const double A0 = rec[8];
  /* low-pass disc, which also holds the centre c itself */
  const double qx = (cx < x0 ? x0 : (cx > x1 ? x1 : cx)) - cx, qy = (cy < y0 ? y0 : (cy > y1 ? y1 : cy)) - cy;
  if (qx * qx + qy * qy <= 0.5 * k) return 1;
  for (int e = 0; e < 4; ++e) {
    double A, B, C, lo, hi;
    if (e < 2) { /* horizontal edge at y */
      const double dy = (e ? y1 : y0) - cy;
      const double px = dy * bx, py = dy * by, pz = A0 + dy * bz;
      A = ax * ax + ay * ay - k * az * az;
      B = ax * px + ay * py - k * az * pz;
      C = px * px + py * py - k * pz * pz;
      lo = x0 - cx; hi = x1 - cx;
    } else { /* vertical edge at x */
      const double dx = (e == 3 ? x1 : x0) - cx;
      const double px = dx * ax, py = dx * ay, pz = A0 + dx * az;
      A = bx * bx + by * by - k * bz * bz;
      B = bx * px + by * py - k * bz * pz;
      C = px * px + py * py - k * pz * pz;
      lo = y0 - cy; hi = y1 - cy;
    }
    if (quad_has_nonpos(A, B, C, lo, hi)) return 1;
  }
  return 0;
}
