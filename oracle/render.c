/*
 * Oracle, Stage 1: full front-to-back rendering of 2D Gaussian surfels with the
 * joint depth proxy. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Sources in the paper:
 *   Sec. 3.3, Eq. 1   surfel frame H = [s_u t_u, s_v t_v, 0, p_k], R = [t_u, t_v, t_w]
 *   Sec. 3.3, Eq. 2   G(u) = exp(-(u^2 + v^2) / 2)
 *   Sec. 3.3          local (u, v) from the intersection of the pixel ray with the
 *                     surfel plane (the 2DGS ray-splat intersection)
 *   Sec. 3.4, Eq. 3   pinhole projection pi(X) = K [X/Z, Y/Z, 1]^T
 *   Sec. 3.1 Stage 1  w_i = alpha_i T_i, colour C = sum c_i w_i and depth proxy
 *                     D = sum d_i w_i from the same weights
 *   Sec. 2.2          the 2DGS depth ordering is kept
 *
 * Readings where the paper is silent (the 3DGS/2DGS rasterizer conventions):
 *   - alpha = min(0.99, o * Ghat); a surfel with alpha < 1/255 is skipped; the
 *     loop stops before a contribution that would bring T below 1e-4.
 *   - Ghat = max(G(u), exp(-|x - c|^2)): the 2DGS object-space low-pass term with
 *     sigma^2 = 1/2 px^2 around the projected centre c; where it wins, the
 *     contribution's depth is the centre depth p_c.z, otherwise the depth of the
 *     ray-plane intersection.
 *   - order: visible surfels sorted by (key, index), the key being p_c.z as the
 *     tile rasterizer computes it in float32 (or_depth_key).
 *   - a surfel is culled when its quaternion is zero, when 255 o < 1 (it can never
 *     reach alpha = 1/255), when p_c.z <= 0.2 m, or when a corner of the square
 *     |u|, |v| <= r_c around its support is not in front of that near plane.
 *   - colour: max(0, 0.5 + sum_lm c_lm Y_lm(dir)) per channel with dir the unit
 *     vector from the camera centre to p_k (real SH, degree <= 3).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int or_quat_to_rot(const float q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double nn = w * w + x * x + y * y + z * z;
  if (!(nn > 0.0)) return 0;
  double inv = 1.0 / sqrt(nn);
  w *= inv; x *= inv; y *= inv; z *= inv;
  /* rotation of a unit quaternion (w, x, y, z) acting on column vectors */
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
  return 1;
}

void or_sh_basis(int deg, const double d[3], double *Y) {
  /* Real spherical harmonics, normalised to unit L2 norm on the sphere, with the
   * Condon-Shortley sign on the odd-m terms. Each constant is the closed-form
   * sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) factor times the polynomial's own. */
  const double pi = 3.14159265358979323846;
  const double x = d[0], y = d[1], z = d[2];
  Y[0] = 0.5 * sqrt(1.0 / pi);
  if (deg < 1) return;
  const double c1 = sqrt(3.0 / (4.0 * pi));
  Y[1] = -c1 * y;
  Y[2] = c1 * z;
  Y[3] = -c1 * x;
  if (deg < 2) return;
  const double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
  Y[4] = c2a * x * y;
  Y[5] = -c2a * y * z;
  Y[6] = c2b * (2 * z * z - x * x - y * y);
  Y[7] = -c2a * x * z;
  Y[8] = c2c * (x * x - y * y);
  if (deg < 3) return;
  const double c3a = 0.25 * sqrt(35.0 / (2 * pi)), c3b = 0.5 * sqrt(105.0 / pi),
               c3c = 0.25 * sqrt(21.0 / (2 * pi)), c3d = 0.25 * sqrt(7.0 / pi),
               c3e = 0.25 * sqrt(105.0 / pi);
  Y[9] = -c3a * y * (3 * x * x - y * y);
  Y[10] = c3b * x * y * z;
  Y[11] = -c3c * y * (4 * z * z - x * x - y * y);
  Y[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
  Y[13] = -c3c * x * (4 * z * z - x * x - y * y);
  Y[14] = c3e * z * (x * x - y * y);
  Y[15] = -c3a * x * (x * x - 3 * y * y);
}

static void project(const or_cam *cam, const double X[3], double *u, double *v) {
  /* Eq. 3 */
  *u = cam->fx * X[0] / X[2] + cam->cx;
  *v = cam->fy * X[1] / X[2] + cam->cy;
}

/* 3D Gaussian (ellipsoid) variant, the 3DGS backbone the method also accepts
 * (Sec. 3.2: any Gaussian splatting variant with per-pixel depth), in the EWA
 * splatting convention of the 3DGS rasterizer: world covariance
 * Sigma = Rq diag(s^2) Rq^T; camera covariance W Sigma W^T with W = R^T (the
 * world-to-camera rotation); screen covariance J (W Sigma W^T) J^T + 0.3 I with
 * the perspective Jacobian J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] at
 * the centre (not clamped); alpha = o exp(-d^T Sigma2D^-1 d / 2); the depth of a
 * contribution is the centre depth. */
static void prepare_ellipsoid(const or_scene *sc, const or_pose *pose, const or_cam *cam, int i, or_splat *s) {
  double Rq[9];
  if (!or_quat_to_rot(sc->quat + 4 * (size_t)i, Rq)) return;
  const double o = sc->opacity[i];
  if (!(255.0 * o >= 1.0)) return;
  const double *R = pose->R, *t = pose->t;
  const double p[3] = {sc->pos[4 * (size_t)i], sc->pos[4 * (size_t)i + 1], sc->pos[4 * (size_t)i + 2]};
  const double dp[3] = {p[0] - t[0], p[1] - t[1], p[2] - t[2]};
  double pc[3];
  for (int k = 0; k < 3; ++k) pc[k] = R[0 * 3 + k] * dp[0] + R[1 * 3 + k] * dp[1] + R[2 * 3 + k] * dp[2];
  if (!(pc[2] > OR_Z_NEAR)) return;
  const float *sv = sc->scale + 4 * (size_t)i;
  const double s2[3] = {(double)sv[0] * sv[0], (double)sv[1] * sv[1], (double)sv[2] * sv[2]};
  /* camera-frame axes of the ellipsoid: A = R^T Rq, covariance A diag(s^2) A^T */
  double A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r * 3 + c] = R[0 * 3 + r] * Rq[0 * 3 + c] + R[1 * 3 + r] * Rq[1 * 3 + c] +
                                            R[2 * 3 + r] * Rq[2 * 3 + c];
  double V[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      V[r * 3 + c] = A[r * 3 + 0] * s2[0] * A[c * 3 + 0] + A[r * 3 + 1] * s2[1] * A[c * 3 + 1] +
                     A[r * 3 + 2] * s2[2] * A[c * 3 + 2];
  const double z = pc[2];
  const double J[6] = {cam->fx / z, 0.0, -cam->fx * pc[0] / (z * z), 0.0, cam->fy / z, -cam->fy * pc[1] / (z * z)};
  double JV[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) JV[r * 3 + c] = J[r * 3 + 0] * V[0 * 3 + c] + J[r * 3 + 1] * V[1 * 3 + c] +
                                             J[r * 3 + 2] * V[2 * 3 + c];
  const double cxx = JV[0] * J[0] + JV[1] * J[1] + JV[2] * J[2] + 0.3;
  const double cxy = JV[0] * J[3] + JV[1] * J[4] + JV[2] * J[5];
  const double cyy = JV[3] * J[3] + JV[4] * J[4] + JV[5] * J[5] + 0.3;
  const double det = cxx * cyy - cxy * cxy;
  if (!(det > 0.0)) return;
  s->prim = 1;
  s->conic[0] = cyy / det;
  s->conic[1] = -cxy / det;
  s->conic[2] = cxx / det;
  s->opacity = o;
  s->rc2 = 2.0 * log(255.0 * o); /* d^T conic d <= rc2  <=>  alpha >= 1/255 */
  project(cam, pc, &s->cx, &s->cy);
  const double ex = sqrt(s->rc2 * cxx), ey = sqrt(s->rc2 * cyy); /* the support ellipse's half extents */
  const double eps = 1e-6;
  s->box[0] = s->cx - ex - eps; s->box[1] = s->cx + ex + eps;
  s->box[2] = s->cy - ey - eps; s->box[3] = s->cy + ey + eps;
  for (int k = 0; k < 3; ++k) s->pc[k] = pc[k];
  double dir[3] = {dp[0], dp[1], dp[2]};
  const double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  for (int k = 0; k < 3; ++k) dir[k] /= dn;
  double Y[16];
  const int deg = sc->sh_degree, K = (deg + 1) * (deg + 1);
  or_sh_basis(deg, dir, Y);
  const float *c = sc->sh + (size_t)i * K * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.5;
    for (int k = 0; k < K; ++k) acc += Y[k] * c[k * 3 + ch];
    s->rgb[ch] = acc > 0.0 ? acc : 0.0;
  }
  s->key = or_depth_key(pose, sc->pos + 4 * (size_t)i);
  s->visible = 1;
}

/* The depth-order key (the 2DGS ordering the method keeps, Sec. 2.2 and
 * Sec. 3.1): the camera depth of the centre as the tile rasterizer computes it,
 * in float32: the world -> camera rotation's last row and offset are rounded to
 * float32 from their FP64 values, and z = r20 x + r21 y + r22 z + t2 is
 * evaluated with one fused multiply-add per term. Evaluating it in float64
 * instead would order surfels whose depths lie a few float32 ulps apart
 * differently from the rasterizer whose order the method defines. */
float or_depth_key(const or_pose *pose, const float p[3]) {
  const double *R = pose->R, *t = pose->t;
  double t2 = 0.0;
  for (int j = 0; j < 3; ++j) t2 = fma(-R[j * 3 + 2], t[j], t2);
  const float r0 = (float)R[0 * 3 + 2], r1 = (float)R[1 * 3 + 2], r2 = (float)R[2 * 3 + 2];
  return fmaf(r0, p[0], fmaf(r1, p[1], fmaf(r2, p[2], (float)t2)));
}

static void prepare_one(const or_scene *sc, const or_pose *pose, const or_cam *cam, int i,
                        or_splat *s) {
  memset(s, 0, sizeof(*s));
  if (sc->primitive == 1) {
    prepare_ellipsoid(sc, pose, cam, i, s);
    return;
  }
  double Rq[9];
  if (!or_quat_to_rot(sc->quat + 4 * (size_t)i, Rq)) return;
  const double o = sc->opacity[i];
  if (!(255.0 * o >= 1.0)) return;
  const double *R = pose->R, *t = pose->t;
  const double p[3] = {sc->pos[4 * (size_t)i], sc->pos[4 * (size_t)i + 1], sc->pos[4 * (size_t)i + 2]};
  const double dp[3] = {p[0] - t[0], p[1] - t[1], p[2] - t[2]};
  double pc[3], tuc[3], tvc[3];
  const double tu[3] = {Rq[0], Rq[3], Rq[6]}, tv[3] = {Rq[1], Rq[4], Rq[7]};
  for (int k = 0; k < 3; ++k) { /* camera frame: X = R^T (P - t) (Eq. 5 with the surfel's own points) */
    pc[k] = R[0 * 3 + k] * dp[0] + R[1 * 3 + k] * dp[1] + R[2 * 3 + k] * dp[2];
    tuc[k] = R[0 * 3 + k] * tu[0] + R[1 * 3 + k] * tu[1] + R[2 * 3 + k] * tu[2];
    tvc[k] = R[0 * 3 + k] * tv[0] + R[1 * 3 + k] * tv[1] + R[2 * 3 + k] * tv[2];
  }
  if (!(pc[2] > OR_Z_NEAR)) return;
  const double su = sc->scale[2 * (size_t)i], sv = sc->scale[2 * (size_t)i + 1];
  for (int r = 0; r < 3; ++r) {
    s->M[r * 3 + 0] = su * tuc[r];
    s->M[r * 3 + 1] = sv * tvc[r];
    s->M[r * 3 + 2] = pc[r];
  }
  s->opacity = o;
  s->rc2 = 2.0 * log(255.0 * o);
  s->lp2 = log(255.0 * o);
  const double rc = sqrt(s->rc2);
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (int c = 0; c < 4; ++c) {
    const double a = (c & 1) ? rc : -rc, b = (c & 2) ? rc : -rc;
    double X[3];
    for (int r = 0; r < 3; ++r) X[r] = pc[r] + a * s->M[r * 3 + 0] + b * s->M[r * 3 + 1];
    if (!(X[2] > OR_Z_NEAR)) return;
    double u, v;
    project(cam, X, &u, &v);
    xmin = fmin(xmin, u); xmax = fmax(xmax, u);
    ymin = fmin(ymin, v); ymax = fmax(ymax, v);
  }
  project(cam, pc, &s->cx, &s->cy);
  const double lp = sqrt(s->lp2);
  xmin = fmin(xmin, s->cx - lp); xmax = fmax(xmax, s->cx + lp);
  ymin = fmin(ymin, s->cy - lp); ymax = fmax(ymax, s->cy + lp);
  const double eps = 1e-6;
  s->box[0] = xmin - eps; s->box[1] = xmax + eps; s->box[2] = ymin - eps; s->box[3] = ymax + eps;
  for (int k = 0; k < 3; ++k) s->pc[k] = pc[k];
  s->su = su;
  s->sv = sv;
  s->pscale = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) + sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  /* view-dependent colour from the camera centre t towards p_k */
  double dir[3] = {dp[0], dp[1], dp[2]};
  const double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  for (int k = 0; k < 3; ++k) dir[k] /= dn;
  double Y[16];
  const int deg = sc->sh_degree, K = (deg + 1) * (deg + 1);
  or_sh_basis(deg, dir, Y);
  const float *c = sc->sh + (size_t)i * K * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.5;
    for (int k = 0; k < K; ++k) acc += Y[k] * c[k * 3 + ch];
    s->rgb[ch] = acc > 0.0 ? acc : 0.0;
  }
  s->key = or_depth_key(pose, sc->pos + 4 * (size_t)i);
  s->visible = 1;
}

void or_prepare(const or_scene *sc, const or_pose *pose, const or_cam *cam, or_splat *out) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < sc->n; ++i) prepare_one(sc, pose, cam, i, &out[i]);
}

static double det3(const double *a, const double *b, const double *c) {
  /* determinant of the 3x3 matrix with columns a, b, c */
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - b[0] * (a[1] * c[2] - a[2] * c[1]) +
         c[0] * (a[1] * b[2] - a[2] * b[1]);
}

double or_eval(const or_splat *s, const or_cam *cam, double x, double y, double *depth,
               double *rho3_out, double *rho2_out) {
  /* Pixel ray r = K^{-1} (x, y, 1) in the camera frame. The surfel point with local
   * coordinates (u, v) is M (u, v, 1); it lies on the ray at depth lambda when
   * M (u, v, 1) = lambda r, i.e. (a, b, g) = M^{-1} r with u = a/g, v = b/g,
   * lambda = 1/g. Solved by Cramer's rule. */
  if (s->prim == 1) { /* ellipsoid: the screen-space Gaussian, centre depth */
    const double dx = x - s->cx, dy = y - s->cy;
    const double rho = s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy + s->conic[2] * dy * dy;
    if (depth) *depth = s->pc[2];
    if (rho3_out) *rho3_out = rho;
    if (rho2_out) *rho2_out = INFINITY;
    return s->opacity * exp(-0.5 * rho);
  }
  const double r[3] = {(x - cam->cx) / cam->fx, (y - cam->cy) / cam->fy, 1.0};
  const double c0[3] = {s->M[0], s->M[3], s->M[6]};
  const double c1[3] = {s->M[1], s->M[4], s->M[7]};
  const double c2[3] = {s->M[2], s->M[5], s->M[8]};
  const double det = det3(c0, c1, c2);
  double rho3 = INFINITY, lam = 0.0;
  if (det != 0.0) {
    const double a = det3(r, c1, c2) / det;
    const double b = det3(c0, r, c2) / det;
    const double g = det3(c0, c1, r) / det;
    if (g > 0.0) {
      const double u = a / g, v = b / g;
      rho3 = u * u + v * v;
      lam = 1.0 / g;
    }
  }
  const double dx = x - s->cx, dy = y - s->cy;
  const double rho2 = 2.0 * (dx * dx + dy * dy); /* low-pass term in the same exponent units */
  const double rho = fmin(rho3, rho2);
  if (depth) *depth = (rho3 <= rho2) ? lam : s->pc[2];
  if (rho3_out) *rho3_out = rho3;
  if (rho2_out) *rho2_out = rho2;
  return s->opacity * exp(-0.5 * rho);
}

/* First-order bound on the error of rho3 = u^2 + v^2 when the intersection is
 * evaluated in float32 (the reading of the tolerance's scope: a float32
 * evaluation of the blend). The solve's inputs carry float32 rounding: the
 * camera-frame centre p_c about c u (|P| + |t|) (a float32 camera transform),
 * the tangent columns and the ray relative c u. Moving the plane by dP moves
 * the intersection along the plane by up to dP (1 + G), G = |n| |r| / |n . r|
 * the inverse cosine between the ray and the normal n = m0 x m1 (large for a
 * surfel seen nearly edge-on), and (u, v) by that over the shorter column;
 * then d rho3 <= 2 sqrt(rho3) d(u, v) + d(u, v)^2. */
#define OR_U (1.0 / 16777216.0) /* float32 unit roundoff */
#define OR_RHO_C 1.0
double or_rho3_err(const or_splat *s, const or_cam *cam, double x, double y, double rho3, double lam) {
  if (s->prim != 0 || !isfinite(rho3)) return 0.0;
  const double r[3] = {(x - cam->cx) / cam->fx, (y - cam->cy) / cam->fy, 1.0};
  const double m0[3] = {s->M[0], s->M[3], s->M[6]}, m1[3] = {s->M[1], s->M[4], s->M[7]};
  const double n[3] = {m0[1] * m1[2] - m0[2] * m1[1], m0[2] * m1[0] - m0[0] * m1[2], m0[0] * m1[1] - m0[1] * m1[0]};
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const double nr = fabs(n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
  const double smin = fmin(s->su, s->sv);
  if (!(nr > 0.0) || !(smin > 0.0)) return INFINITY;
  const double G = nn * rn / nr;
  const double q = sqrt(rho3);
  const double dP = OR_RHO_C * OR_U * (s->pscale + q * (s->su + s->sv) + lam * rn);
  const double duv = dP * (1.0 + G) / smin;
  return 2.0 * q * duv + duv * duv;
}

typedef struct {
  float key;
  int idx;
} order_item;

static int cmp_item(const void *pa, const void *pb) {
  const order_item *a = (const order_item *)pa, *b = (const order_item *)pb;
  if (a->key < b->key) return -1;
  if (a->key > b->key) return 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

static int *depth_order(const or_splat *sp, int n, int *nvis) {
  order_item *items = (order_item *)malloc(sizeof(order_item) * (size_t)(n > 0 ? n : 1));
  int m = 0;
  for (int i = 0; i < n; ++i)
    if (sp[i].visible) { items[m].key = sp[i].key; items[m].idx = i; ++m; }
  qsort(items, (size_t)m, sizeof(order_item), cmp_item);
  int *ord = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  for (int k = 0; k < m; ++k) ord[k] = items[k].idx;
  free(items);
  *nvis = m;
  return ord;
}

static uint32_t fbits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* Front-to-back blend of one pixel over all visible surfels in depth order. */
/* A first-order bound on how far a float32 evaluation of the same blending sum
 * can be from the exact one at this pixel (u = 2^-24). Two parts:
 *  - rounding of the blend itself: alpha carries a relative error of about
 *    3u + 4u rho (the exponential and its argument; none once clamped at 0.99),
 *    and through (1 - alpha) each factor of the running transmittance adds
 *    2u + alpha / (1 - alpha) times that error; every weight alpha T then carries
 *    the errors of its alpha and of its T, each colour about 20u of its magnitude
 *    (at least 0.5), and the n-term sum nu of the total;
 *  - the conditioning of the ray-plane solve: alpha_k moves by alpha_k e_k,
 *    e_k = half the float32 error of rho3 (or_rho3_err) where that term decides,
 *    and the colour moves by dC/dalpha_k = T_k c_k - C_behind_k / (1 - alpha_k)
 *    times that (C_behind_k: everything blended behind k, the background
 *    included). The largest of these terms enters: the surfels' roundings are
 *    independent, and their worst cases summed over a pixel's contributors
 *    overstate a float32 evaluation's error ten to twenty times on 3M-surfel
 *    scenes, while a pixel where one surfel alone can move the colour past the
 *    tolerance (a surfel seen nearly edge-on) is what cannot meet it.
 * Used by the tests to tell pixels whose float32 value cannot meet an absolute
 * tolerance by construction from pixels that must. */
#define OR_MAX_CONTRIB 2560 /* T >= 1e-4 with alpha >= 1/255 allows at most 2345 */
static void render_pixel(const or_splat *sp, const int *ord, int nvis, const or_cam *cam,
                         const double bg[3], double x, double y, double out_rgb[3],
                         double *out_d, double *out_t, double *out_margin, int64_t *out_pairs,
                         double *out_bound, double (*ck)[6]) {
  double T = 1.0, C[3] = {0, 0, 0}, D = 0.0, mrg = INFINITY;
  double eT = 0.0, bnd = 0.0, cabs = 0.0;
  int ncontrib = 0;
  int64_t pairs = 0;
  int have_prev = 0;
  float prev_key = 0.f;
  double prev_w = 0.0;
  /* ck (scratch of OR_MAX_CONTRIB rows, with the bound): per contributor T, alpha,
   * the alpha error of the solve's conditioning, colour */
  if (!out_bound) ck = NULL;
  for (int k = 0; k < nvis; ++k) {
    const or_splat *s = &sp[ord[k]];
    if (x < s->box[0] || x > s->box[1] || y < s->box[2] || y > s->box[3]) continue;
    double dep, rho3, rho2;
    const double oG = or_eval(s, cam, x, y, &dep, &rho3, &rho2);
    ++pairs;
    /* float32 error of rho3, and of rho = min(rho3, rho2) (rho3 may dip below
     * the low-pass term by that much); only with the bound requested */
    const double erho3 = out_bound ? or_rho3_err(s, cam, x, y, rho3, dep) : 0.0;
    const double erho = rho3 <= rho2 ? erho3 : fmax(0.0, erho3 - (rho3 - rho2));
    const double rho = isfinite(rho3) ? fmin(rho3, rho2) : rho2;
    /* margins of the skip and stop decisions, at any transmittance: a flip adds
     * or drops a weight alpha T, and a deep surfel behind a near one moves the
     * depth proxy by alpha T d, relatively more than the colour. The skip
     * threshold alpha = 1/255 is rho = rc2: the decision is only safe when rho
     * lies farther from rc2 than its float32 error (in the same relative units:
     * half the rho gap). */
    mrg = fmin(mrg, fabs(oG * 255.0 - 1.0));
    if (erho > 0.0) mrg = fmin(mrg, 0.5 * (fabs(rho - s->rc2) - erho));
    const double a = oG < OR_ALPHA_MAX ? oG : OR_ALPHA_MAX;
    if (a < OR_ALPHA_MIN) continue;
    const double ea = a < OR_ALPHA_MAX ? OR_U * (3.0 + 4.0 * rho) : 0.0;
    const double ec = a < OR_ALPHA_MAX ? 0.5 * erho : 0.0;
    const double Tn = T * (1.0 - a);
    /* with the bound requested, T's own float32 error narrows the stop margin */
    mrg = fmin(mrg, fabs(Tn - OR_T_MIN) / OR_T_MIN - (out_bound ? eT + a / (1.0 - a) * (ea + ec) : 0.0));
    if (Tn < OR_T_MIN) break;
    const double w = a * T;
    if (isfinite(rho3) && w * fabs(dep - s->pc[2]) > 1e-5 * s->pc[2])
      mrg = fmin(mrg, (fabs(rho3 - rho2) - erho3) / fmax(rho3, rho2));
    if (have_prev && w > 1e-3 && prev_w > 1e-3) {
      const uint32_t kb = fbits(s->key), pb = fbits(prev_key);
      const uint32_t du = kb > pb ? kb - pb : pb - kb;
      if (du <= 2) mrg = 0.0; /* near-equal depth keys: the order may differ in float32 */
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] += w * s->rgb[ch];
    D += w * dep;
    const double cm = fmax(fmax(fabs(s->rgb[0]), fabs(s->rgb[1])), fabs(s->rgb[2]));
    bnd += w * (cm * (eT + ea + OR_U) + 20.0 * OR_U * fmax(cm, 0.5));
    cabs += w * cm;
    /* the transmittance's relative error: rounding, and the conditioning errors
     * of the alphas in front (those also enter through the per-alpha sum below) */
    eT += 2.0 * OR_U + a / (1.0 - a) * (ea + ec);
    if (ck && ncontrib < OR_MAX_CONTRIB) {
      ck[ncontrib][0] = T;
      ck[ncontrib][1] = a;
      ck[ncontrib][2] = ec;
      for (int ch = 0; ch < 3; ++ch) ck[ncontrib][3 + ch] = s->rgb[ch];
    }
    T = Tn;
    have_prev = 1; prev_key = s->key; prev_w = w;
    ++ncontrib;
  }
  for (int ch = 0; ch < 3; ++ch) out_rgb[ch] = C[ch] + T * (bg ? bg[ch] : 0.0);
  *out_d = D;
  *out_t = T;
  if (out_margin) *out_margin = mrg;
  if (out_pairs) *out_pairs = pairs;
  if (out_bound) {
    /* the conditioning part: back to front, C_behind accumulates */
    double cb[3] = {T * (bg ? bg[0] : 0.0), T * (bg ? bg[1] : 0.0), T * (bg ? bg[2] : 0.0)}, cond = 0.0;
    const int nk = ncontrib < OR_MAX_CONTRIB ? ncontrib : OR_MAX_CONTRIB;
    for (int k = nk - 1; k >= 0; --k) {
      const double Tk = ck[k][0], ak = ck[k][1], eck = ck[k][2];
      double sens = 0.0;
      for (int ch = 0; ch < 3; ++ch) sens = fmax(sens, fabs(Tk * ck[k][3 + ch] - cb[ch] / (1.0 - ak)));
      cond = fmax(cond, sens * ak * eck);
      for (int ch = 0; ch < 3; ++ch) cb[ch] += Tk * ak * ck[k][3 + ch];
    }
    *out_bound = bnd + ncontrib * OR_U * cabs + cond;
  }
}

int or_render(const or_scene *sc, const or_pose *pose, const or_cam *cam, const double bg[3],
              int x0, int y0, int w, int h, double *rgb, double *depth, double *trans,
              double *margin, int64_t *pairs, double *fp32_bound) {
  if (!sc || !pose || !cam || w < 0 || h < 0 || sc->n < 0) return -1;
  or_splat *sp = (or_splat *)malloc(sizeof(or_splat) * (size_t)(sc->n > 0 ? sc->n : 1));
  or_prepare(sc, pose, cam, sp);
  int nvis = 0;
  int *ord = depth_order(sp, sc->n, &nvis);
  /* only surfels whose box meets the window can pass a pixel's box test (the
   * depth order is kept) */
  int nwin = 0;
  for (int k = 0; k < nvis; ++k) {
    const double *b = sp[ord[k]].box;
    if (b[1] >= x0 && b[0] <= x0 + w - 1 && b[3] >= y0 && b[2] <= y0 + h - 1) ord[nwin++] = ord[k];
  }
  const size_t npix = (size_t)w * h;
  int64_t total = 0;
#pragma omp parallel reduction(+ : total)
  {
    double (*ck)[6] = fp32_bound ? (double (*)[6])malloc(sizeof(double[6]) * OR_MAX_CONTRIB) : NULL;
#pragma omp for schedule(dynamic, 1)
    for (int j = 0; j < h; ++j) {
      for (int i = 0; i < w; ++i) {
        const size_t p = (size_t)j * w + i;
        double c3[3], m;
        int64_t np;
        render_pixel(sp, ord, nwin, cam, bg, (double)(x0 + i), (double)(y0 + j), c3, &depth[p],
                     &trans[p], &m, &np, fp32_bound ? &fp32_bound[p] : NULL, ck);
        for (int ch = 0; ch < 3; ++ch) rgb[ch * npix + p] = c3[ch];
        if (margin) margin[p] = m;
        total += np;
      }
    }
    free(ck);
  }
  if (pairs) *pairs = total;
  free(ord);
  free(sp);
  return nvis;
}

int or_render_tiles(const or_scene *sc, const or_pose *pose, const or_cam *cam, const double bg[3],
                    int tile, const uint8_t *tile_mask, double *rgb, double *depth, double *trans) {
  if (!sc || !pose || !cam || tile <= 0) return -1;
  or_splat *sp = (or_splat *)malloc(sizeof(or_splat) * (size_t)(sc->n > 0 ? sc->n : 1));
  or_prepare(sc, pose, cam, sp);
  int nvis = 0;
  int *ord = depth_order(sp, sc->n, &nvis);
  const int W = cam->W, H = cam->H, tx = (W + tile - 1) / tile;
  const size_t npix = (size_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      if (!tile_mask[(y / tile) * tx + (x / tile)]) continue;
      const size_t p = (size_t)y * W + x;
      double c3[3];
      render_pixel(sp, ord, nvis, cam, bg, (double)x, (double)y, c3, &depth[p], &trans[p], NULL,
                   NULL, NULL, NULL);
      for (int ch = 0; ch < 3; ++ch) rgb[ch * npix + p] = c3[ch];
    }
  }
  free(ord);
  free(sp);
  return nvis;
}

/* ------------------------------------------------------------------ integer helpers */

int or_tile_rect(const float bounds[4], int W, int H, int tile, int rect[4]) {
  /* pixels whose centres lie inside [xmin, xmax] x [ymin, ymax], clipped to the
   * image, mapped to the tiles that contain them */
  const double xmin = bounds[0], xmax = bounds[1], ymin = bounds[2], ymax = bounds[3];
  rect[0] = rect[1] = 0;
  rect[2] = rect[3] = -1;
  if (!(xmax >= 0.0) || !(ymax >= 0.0) || !(xmin <= W - 1.0) || !(ymin <= H - 1.0)) return 0;
  const int px0 = xmin <= 0.0 ? 0 : (int)ceil(xmin);
  const int px1 = xmax >= W - 1.0 ? W - 1 : (int)floor(xmax);
  const int py0 = ymin <= 0.0 ? 0 : (int)ceil(ymin);
  const int py1 = ymax >= H - 1.0 ? H - 1 : (int)floor(ymax);
  if (px0 > px1 || py0 > py1) return 0;
  rect[0] = px0 / tile; rect[1] = py0 / tile; rect[2] = px1 / tile; rect[3] = py1 / tile;
  return (rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1);
}

void or_sort_pairs(int64_t n, uint64_t *keys, uint32_t *vals) {
  /* bottom-up merge sort: stable, so equal keys keep their input order */
  if (n <= 1) return;
  uint64_t *k2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  uint32_t *v2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint64_t *ka = keys, *kb = k2;
  uint32_t *va = vals, *vb = v2;
  for (int64_t width = 1; width < n; width *= 2) {
    for (int64_t lo = 0; lo < n; lo += 2 * width) {
      int64_t mid = lo + width < n ? lo + width : n, hi = lo + 2 * width < n ? lo + 2 * width : n;
      int64_t i = lo, j = mid, o = lo;
      while (i < mid && j < hi) {
        if (ka[j] < ka[i]) { kb[o] = ka[j]; vb[o++] = va[j++]; }
        else { kb[o] = ka[i]; vb[o++] = va[i++]; }
      }
      while (i < mid) { kb[o] = ka[i]; vb[o++] = va[i++]; }
      while (j < hi) { kb[o] = ka[j]; vb[o++] = va[j++]; }
    }
    uint64_t *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    memcpy(keys, ka, sizeof(uint64_t) * (size_t)n);
    memcpy(vals, va, sizeof(uint32_t) * (size_t)n);
  }
  free(k2);
  free(v2);
}
