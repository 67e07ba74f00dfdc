/*
 * Oracle, Stages 2-4: depth-guided reprojection, hole categorisation, gap
 * interpolation, the adaptive ROI generator and the composition of the
 * affiliated eye. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sources in the paper:
 *   Sec. 3.1 Stage 2, Sec. 3.4 Eq. 3-5   unproject with the depth proxy, transfer,
 *                                        project into the affiliated eye
 *   Sec. 3.1 Stages 3-4, Sec. 3.5        holes -> gaps (interpolated) and ROIs
 *                                        (targeted re-rendering)
 *   Sec. 3.5 Step 1, Eq. 6-8             edge ROIs from boundary samples at two
 *                                        depth hypotheses, margin m = 32, 16x16 tiles
 *   Sec. 3.5 Step 2                      connected centre holes -> bounding box ->
 *                                        expanded by m -> tile aligned
 *   Sec. 4.3                             ROI regions are re-rasterised
 *
 * Readings where the paper is silent:
 *   - a source pixel is valid when its coverage 1 - T >= 0.5; it warps with the
 *     alpha-normalised depth D / (1 - T). A pixel below that coverage carries
 *     (mostly) background: it is transferred as a sample at infinite depth
 *     (direction only, so a pure translation keeps it in place) and loses every
 *     depth test against a surface sample.
 *   - a source sample lands on pixel (floor(x + 0.5), floor(y + 0.5)) when that is
 *     inside the image and its destination depth is beyond 0.2 m; the smallest
 *     float32 depth wins, ties go to the smaller source linear index.
 *   - edge ROI: N samples per edge at round(k (L-1)/(N-1)); the depth hypotheses
 *     are the per-frame min/max of the normalised depth over valid pixels (or
 *     fixed values); a projected sample counts when its depth is beyond 0.2 m and
 *     is taken at the pixel it rounds to, so (x, y) in Eq. 6 are integers.
 *     With no valid sample every border gets its maximum width.
 *   - gap: a hole outside the edge strips whose maximal horizontal (or vertical)
 *     hole run is at most gap_thresh long and has valid pixels at both ends; it is
 *     filled by linear interpolation between those ends along the shorter such run
 *     (horizontal on a tie). Other holes are centre holes; with the centre step
 *     off they are filled along their row (linear between the nearest valid
 *     pixels, or copied from the only one), else along their column, else 0.
 *   - centre components use 4-connectivity and every component becomes an ROI.
 *   - every pixel of a tile touched by an ROI takes the full affiliated render.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static void mat_t_vec(const double *R, const double *v, double *o) {
  for (int k = 0; k < 3; ++k) o[k] = R[0 * 3 + k] * v[0] + R[1 * 3 + k] * v[1] + R[2 * 3 + k] * v[2];
}

static void mat_vec(const double *R, const double *v, double *o) {
  for (int k = 0; k < 3; ++k) o[k] = R[k * 3 + 0] * v[0] + R[k * 3 + 1] * v[1] + R[k * 3 + 2] * v[2];
}

/* Eq. 4 then Eq. 5 for one source pixel (x, y). depth > 0: a surface sample at
 * that depth; depth = +inf: a background sample (direction only). Returns 1 and
 * the destination coordinates and depth when the point is in front of the
 * destination near plane. */
static int transfer(const or_cam *cam, const or_pose *src, const or_pose *dst, double x, double y,
                    double depth, double *u, double *v, double *z) {
  const double ray[3] = {(x - cam->cx) / cam->fx, (y - cam->cy) / cam->fy, 1.0}; /* pi^{-1}(u, 1) */
  double Xd[3];
  if (isinf(depth)) {
    double w[3];
    mat_vec(src->R, ray, w);
    mat_t_vec(dst->R, w, Xd);
    if (!(Xd[2] > 0.0)) return 0;
    *z = INFINITY;
  } else {
    const double Xs[3] = {ray[0] * depth, ray[1] * depth, depth};
    double P[3];
    mat_vec(src->R, Xs, P);
    for (int k = 0; k < 3; ++k) P[k] += src->t[k]; /* Eq. 4 */
    const double d[3] = {P[0] - dst->t[0], P[1] - dst->t[1], P[2] - dst->t[2]};
    mat_t_vec(dst->R, d, Xd); /* Eq. 5 */
    if (!(Xd[2] > OR_Z_NEAR)) return 0;
    *z = Xd[2];
  }
  *u = cam->fx * Xd[0] / Xd[2] + cam->cx; /* Eq. 3 */
  *v = cam->fy * Xd[1] / Xd[2] + cam->cy;
  return 1;
}

static double round_margin(double c) {
  const double f = (c + 0.5) - floor(c + 0.5);
  return f < 1.0 - f ? f : 1.0 - f;
}

void or_warp(const or_cam *cam, const or_pose *src, const or_pose *dst, const double *rgb,
             const double *D, const double *T, int64_t *tgt, float *zkey, double *tmargin,
             int64_t *winner, float *zdst, double *out_rgb, uint8_t *hole) {
  const int W = cam->W, H = cam->H;
  const int64_t npix = (int64_t)W * H;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npix; ++i) {
    const int x = (int)(i % W), y = (int)(i / W);
    const double cov = 1.0 - T[i];
    const double depth = cov >= 0.5 ? D[i] / cov : INFINITY;
    double u, v, z;
    tgt[i] = -1;
    zkey[i] = INFINITY;
    tmargin[i] = INFINITY;
    if (!transfer(cam, src, dst, x, y, depth, &u, &v, &z)) continue;
    const double fx = floor(u + 0.5), fy = floor(v + 0.5);
    if (!(fx >= 0.0 && fx <= W - 1.0 && fy >= 0.0 && fy <= H - 1.0)) continue;
    tgt[i] = (int64_t)fy * W + (int64_t)fx;
    zkey[i] = (float)z;
    const double mu = round_margin(u), mv = round_margin(v);
    tmargin[i] = mu < mv ? mu : mv;
  }
  for (int64_t p = 0; p < npix; ++p) { winner[p] = -1; zdst[p] = INFINITY; }
  /* depth test: smallest key wins, the first (smallest) source index on ties */
  for (int64_t i = 0; i < npix; ++i) {
    const int64_t p = tgt[i];
    if (p < 0) continue;
    if (winner[p] < 0 || zkey[i] < zdst[p]) { winner[p] = i; zdst[p] = zkey[i]; }
  }
  for (int64_t p = 0; p < npix; ++p) {
    hole[p] = winner[p] < 0;
    for (int ch = 0; ch < 3; ++ch) out_rgb[ch * npix + p] = winner[p] < 0 ? 0.0 : rgb[ch * npix + winner[p]];
  }
}

int64_t or_depth_range(int npix, const double *D, const double *T, double *dmin, double *dmax) {
  double lo = INFINITY, hi = -INFINITY;
  int64_t cnt = 0;
  for (int i = 0; i < npix; ++i) {
    const double cov = 1.0 - T[i];
    if (!(cov >= 0.5)) continue;
    const double d = D[i] / cov;
    lo = d < lo ? d : lo;
    hi = d > hi ? d : hi;
    ++cnt;
  }
  *dmin = lo;
  *dmax = hi;
  return cnt;
}

static int clampi(int x, int a, int b) { return x < a ? a : (x > b ? b : x); }

void or_edge_roi(const or_cam *cam, const or_pose *src, const or_pose *dst, int nsamples,
                 double dmin, double dmax, int m, int tile, int widths[4], int strips[16],
                 double *margin) {
  const int W = cam->W, H = cam->H, N = nsamples;
  long xmin = 0, xmax = 0, ymin = 0, ymax = 0;
  int any = 0;
  double mrg = INFINITY;
  const double depths[2] = {dmin, dmax};
  for (int e = 0; e < 4; ++e) {
    for (int k = 0; k < N; ++k) {
      int x, y;
      const int along = (e < 2) ? W : H;
      /* round(k (L-1)/(N-1)) in integer arithmetic */
      const int pos = (int)(((long)2 * k * (along - 1) + (N - 1)) / (2L * (N - 1)));
      if (e == 0) { x = pos; y = 0; }          /* top edge */
      else if (e == 1) { x = pos; y = H - 1; } /* bottom edge */
      else if (e == 2) { x = 0; y = pos; }     /* left edge */
      else { x = W - 1; y = pos; }             /* right edge */
      for (int d = 0; d < 2; ++d) {
        double u, v, z;
        if (!(depths[d] > 0.0) || !transfer(cam, src, dst, x, y, depths[d], &u, &v, &z)) continue;
        u = fmax(-1e9, fmin(1e9, u)); /* keeps the integer conversion defined */
        v = fmax(-1e9, fmin(1e9, v));
        const long px = (long)floor(u + 0.5), py = (long)floor(v + 0.5);
        const double mu = round_margin(u), mv = round_margin(v);
        mrg = fmin(mrg, fmin(mu, mv));
        if (!any) { xmin = xmax = px; ymin = ymax = py; any = 1; }
        else {
          xmin = px < xmin ? px : xmin; xmax = px > xmax ? px : xmax;
          ymin = py < ymin ? py : ymin; ymax = py > ymax ? py : ymax;
        }
      }
    }
  }
  int lw, rw, th, bh;
  if (!any) { lw = rw = W / 2; th = bh = H / 2; }
  else {
    /* Eq. 7, Eq. 8 and their vertical analogues; ceil/floor are identities on the
     * integer sample positions */
    lw = xmin > 0 ? clampi((int)(xmin > W ? W : xmin) + m, 0, W / 2) : 0;
    rw = xmax < W - 1 ? clampi((int)((W - 1) - (xmax < -1 ? -1 : xmax)) + m, 0, W / 2) : 0;
    th = ymin > 0 ? clampi((int)(ymin > H ? H : ymin) + m, 0, H / 2) : 0;
    bh = ymax < H - 1 ? clampi((int)((H - 1) - (ymax < -1 ? -1 : ymax)) + m, 0, H / 2) : 0;
  }
  widths[0] = lw; widths[1] = rw; widths[2] = th; widths[3] = bh;
  /* tile-aligned strips, outward: left, right, top, bottom */
  int *s = strips;
  const int lx1 = lw > 0 ? (lw + tile - 1) / tile * tile : 0;
  s[0] = 0; s[1] = 0; s[2] = lx1 < W ? lx1 : W; s[3] = lw > 0 ? H : 0;
  const int rx0 = rw > 0 ? (W - rw) / tile * tile : W;
  s[4] = rx0; s[5] = 0; s[6] = W; s[7] = rw > 0 ? H : 0;
  const int ty1 = th > 0 ? (th + tile - 1) / tile * tile : 0;
  s[8] = 0; s[9] = 0; s[10] = th > 0 ? W : 0; s[11] = ty1 < H ? ty1 : H;
  const int by0 = bh > 0 ? (H - bh) / tile * tile : H;
  s[12] = 0; s[13] = by0; s[14] = bh > 0 ? W : 0; s[15] = H;
  if (margin) *margin = mrg;
}

void or_classify(int W, int H, const uint8_t *hole, const double *rgb_in, const uint8_t *in_strip,
                 int gap_thresh, int center_enabled, uint8_t *cls, double *rgb_out) {
  const int64_t npix = (int64_t)W * H;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < npix; ++p) {
    const int x = (int)(p % W), y = (int)(p / W);
    uint8_t c = 0;
    if (hole[p]) c |= OR_CLS_HOLE;
    if (in_strip[p]) c |= OR_CLS_STRIP;
    for (int ch = 0; ch < 3; ++ch) rgb_out[ch * npix + p] = hole[p] ? 0.0 : rgb_in[ch * npix + p];
    if (!hole[p] || in_strip[p]) { cls[p] = c; continue; }
    /* maximal horizontal and vertical hole runs through p */
    int a = x, b = x;
    while (a - 1 >= 0 && hole[p - (x - (a - 1))]) --a;
    while (b + 1 <= W - 1 && hole[p + (b + 1 - x)]) ++b;
    int at = y, bt = y;
    while (at - 1 >= 0 && hole[(int64_t)(at - 1) * W + x]) --at;
    while (bt + 1 <= H - 1 && hole[(int64_t)(bt + 1) * W + x]) ++bt;
    const int Lh = b - a + 1, Lv = bt - at + 1;
    const int bnd_h = a - 1 >= 0 && b + 1 <= W - 1; /* ends are valid by maximality */
    const int bnd_v = at - 1 >= 0 && bt + 1 <= H - 1;
    const int gap_h = bnd_h && Lh <= gap_thresh, gap_v = bnd_v && Lv <= gap_thresh;
    int axis = -1; /* 0 horizontal, 1 vertical */
    if (gap_h && gap_v) axis = Lv < Lh ? 1 : 0;
    else if (gap_h) axis = 0;
    else if (gap_v) axis = 1;
    if (axis >= 0) {
      c |= OR_CLS_GAP;
      const int64_t e0 = axis == 0 ? (int64_t)y * W + (a - 1) : (int64_t)(at - 1) * W + x;
      const int64_t e1 = axis == 0 ? (int64_t)y * W + (b + 1) : (int64_t)(bt + 1) * W + x;
      const double span = axis == 0 ? (double)(b + 1 - (a - 1)) : (double)(bt + 1 - (at - 1));
      const double tpos = axis == 0 ? (double)(x - (a - 1)) / span : (double)(y - (at - 1)) / span;
      for (int ch = 0; ch < 3; ++ch)
        rgb_out[ch * npix + p] = (1.0 - tpos) * rgb_in[ch * npix + e0] + tpos * rgb_in[ch * npix + e1];
    } else {
      c |= OR_CLS_CENTRE;
      if (!center_enabled) {
        /* fallback fill along the row, else the column */
        const int hasL = a - 1 >= 0, hasR = b + 1 <= W - 1, hasU = at - 1 >= 0, hasD = bt + 1 <= H - 1;
        int64_t e0 = -1, e1 = -1;
        double tpos = 0.0;
        if (hasL || hasR) {
          e0 = hasL ? (int64_t)y * W + (a - 1) : -1;
          e1 = hasR ? (int64_t)y * W + (b + 1) : -1;
          tpos = (double)(x - (a - 1)) / (double)(b + 1 - (a - 1));
        } else if (hasU || hasD) {
          e0 = hasU ? (int64_t)(at - 1) * W + x : -1;
          e1 = hasD ? (int64_t)(bt + 1) * W + x : -1;
          tpos = (double)(y - (at - 1)) / (double)(bt + 1 - (at - 1));
        }
        for (int ch = 0; ch < 3; ++ch) {
          double v = 0.0;
          if (e0 >= 0 && e1 >= 0) v = (1.0 - tpos) * rgb_in[ch * npix + e0] + tpos * rgb_in[ch * npix + e1];
          else if (e0 >= 0) v = rgb_in[ch * npix + e0];
          else if (e1 >= 0) v = rgb_in[ch * npix + e1];
          rgb_out[ch * npix + p] = v;
        }
      }
    }
    cls[p] = c;
  }
}

int or_center_rois(int W, int H, const uint8_t *cls, int m, int tile, int *rects, int cap) {
  const int64_t npix = (int64_t)W * H;
  uint8_t *seen = (uint8_t *)calloc((size_t)(npix > 0 ? npix : 1), 1);
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npix > 0 ? npix : 1));
  const int tx_max = (W + tile - 1) / tile - 1, ty_max = (H + tile - 1) / tile - 1;
  int count = 0;
  for (int64_t s = 0; s < npix; ++s) {
    if (!(cls[s] & OR_CLS_CENTRE) || seen[s]) continue;
    /* breadth-first flood fill of the 4-connected component that starts at s,
     * which is its smallest linear index because s is visited in order */
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    seen[s] = 1;
    int x0 = W, y0 = H, x1 = -1, y1 = -1;
    while (head < tail) {
      const int64_t p = queue[head++];
      const int x = (int)(p % W), y = (int)(p / W);
      x0 = x < x0 ? x : x0; x1 = x > x1 ? x : x1;
      y0 = y < y0 ? y : y0; y1 = y > y1 ? y : y1;
      const int64_t nb[4] = {x > 0 ? p - 1 : -1, x < W - 1 ? p + 1 : -1, y > 0 ? p - W : -1,
                             y < H - 1 ? p + W : -1};
      for (int k = 0; k < 4; ++k) {
        const int64_t q = nb[k];
        if (q >= 0 && (cls[q] & OR_CLS_CENTRE) && !seen[q]) { seen[q] = 1; queue[tail++] = q; }
      }
    }
    if (count < cap) {
      /* expand by m, align outward to the tile grid, clip to the image */
      const int tx0 = (x0 - m) <= 0 ? 0 : (x0 - m) / tile;
      const int ty0 = (y0 - m) <= 0 ? 0 : (y0 - m) / tile;
      int tx1 = (x1 + m) / tile, ty1 = (y1 + m) / tile;
      tx1 = tx1 > tx_max ? tx_max : tx1;
      ty1 = ty1 > ty_max ? ty_max : ty1;
      int *r = rects + 4 * (size_t)count;
      r[0] = tx0 * tile; r[1] = ty0 * tile;
      r[2] = (tx1 + 1) * tile < W ? (tx1 + 1) * tile : W;
      r[3] = (ty1 + 1) * tile < H ? (ty1 + 1) * tile : H;
    }
    ++count;
  }
  free(queue);
  free(seen);
  return count;
}

static void mark_rect_tiles(int W, int H, int tile, const int *r, uint8_t *tile_mask) {
  const int tx = (W + tile - 1) / tile;
  if (r[2] <= r[0] || r[3] <= r[1]) return;
  for (int ty = r[1] / tile; ty <= (r[3] - 1) / tile; ++ty)
    for (int t = r[0] / tile; t <= (r[2] - 1) / tile; ++t) tile_mask[ty * tx + t] = 1;
}

int or_stereo(const or_scene *sc, const or_pose *dom, const or_pose *aff, const or_cam *cam,
              const double bg[3], const or_params *p, double *rgb_dom, double *depth_dom,
              double *trans_dom, double *rgb_aff, uint8_t *cls, int widths[4], int *rects,
              int rect_cap, int *nrects, uint8_t *tile_mask) {
  const int W = cam->W, H = cam->H, tile = p->tile;
  const int64_t npix = (int64_t)W * H;
  if (W <= 0 || H <= 0 || tile <= 0 || p->nsamples < 2) return -1;
  /* Stage 1 */
  or_render(sc, dom, cam, bg, 0, 0, W, H, rgb_dom, depth_dom, trans_dom, NULL, NULL, NULL);
  /* Stage 2 */
  int64_t *tgt = (int64_t *)malloc(sizeof(int64_t) * npix), *win = (int64_t *)malloc(sizeof(int64_t) * npix);
  float *zk = (float *)malloc(sizeof(float) * npix), *zd = (float *)malloc(sizeof(float) * npix);
  double *tm = (double *)malloc(sizeof(double) * npix), *wrgb = (double *)malloc(sizeof(double) * 3 * npix);
  uint8_t *hole = (uint8_t *)malloc(npix), *strip = (uint8_t *)calloc(npix, 1);
  or_warp(cam, dom, aff, rgb_dom, depth_dom, trans_dom, tgt, zk, tm, win, zd, wrgb, hole);
  /* Step 1: edge ROIs */
  double dmin = p->dmin, dmax = p->dmax;
  if (p->depth_mode == 0) or_depth_range((int)npix, depth_dom, trans_dom, &dmin, &dmax);
  int strips[16];
  or_edge_roi(cam, dom, aff, p->nsamples, dmin, dmax, p->margin, tile, widths, strips, NULL);
  const int ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
  memset(tile_mask, 0, (size_t)ntx * nty);
  for (int k = 0; k < 4; ++k) {
    const int *r = strips + 4 * k;
    for (int y = r[1]; y < r[3]; ++y)
      for (int x = r[0]; x < r[2]; ++x) strip[(int64_t)y * W + x] = 1;
    mark_rect_tiles(W, H, tile, r, tile_mask);
  }
  /* Stages 3-4: gaps and centre holes */
  or_classify(W, H, hole, wrgb, strip, p->gap_thresh, p->enable_center, cls, rgb_aff);
  int nc = 0;
  if (p->enable_center) {
    nc = or_center_rois(W, H, cls, p->margin, tile, rects, rect_cap);
    for (int k = 0; k < nc && k < rect_cap; ++k) mark_rect_tiles(W, H, tile, rects + 4 * k, tile_mask);
  }
  *nrects = nc;
  /* targeted rendering of the ROI tiles, composed over the reprojected image */
  double *fr = (double *)calloc(3 * npix, sizeof(double)), *fd = (double *)calloc(npix, sizeof(double)),
         *ft = (double *)calloc(npix, sizeof(double));
  or_render_tiles(sc, aff, cam, bg, tile, tile_mask, fr, fd, ft);
  for (int64_t q = 0; q < npix; ++q) {
    const int x = (int)(q % W), y = (int)(q / W);
    if (!tile_mask[(y / tile) * ntx + x / tile]) continue;
    cls[q] |= OR_CLS_RENDER;
    for (int ch = 0; ch < 3; ++ch) rgb_aff[ch * npix + q] = fr[ch * npix + q];
  }
  free(fr); free(fd); free(ft);
  free(tgt); free(win); free(zk); free(zd); free(tm); free(wrgb); free(hole); free(strip);
  return 0;
}
