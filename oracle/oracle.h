/*
 * FP64 CPU oracle for binocular 2D-Gaussian-surfel rendering by reprojection and
 * selective patching (Zhu & Zhou, "From Mono to Stereo").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline of the benchmark load this library. It shares no code, header, table
 * or constant with the CUDA path; the two are compared on the same seeded inputs.
 *
 * Every function is a plain restatement of the paper's definitions, in double
 * precision, without tiling: a pixel loops over every surfel in depth order.
 * Where the paper is silent the readings are stated beside the code.
 *
 * Conventions shared with the inputs (not with the CUDA code):
 *   scene arrays  pos[n][4] (xyz + pad), quat[n][4] (w,x,y,z), scale[n][2],
 *                 opacity[n], sh[n][(deg+1)^2][3], all float32, host memory
 *   pose          camera-to-world (R row-major, t), P_world = R X_cam + t (Eq. 4)
 *   camera        pinhole K = [[fx,0,cx],[0,fy,cy],[0,0,1]] (Eq. 3); pixel
 *                 centres at integer coordinates 0..W-1, 0..H-1
 *   images        planar: rgb[3][H][W], depth[H][W], trans[H][W]
 */
#ifndef ORACLE_ORACLE_H
#define ORACLE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n;
  int sh_degree;
  const float *pos, *quat, *scale, *opacity, *sh;
  int primitive; /* 0: 2D surfels (scale [n][2]); 1: 3D ellipsoids (scale [n][4]: sx, sy, sz, unused) */
} or_scene;

typedef struct {
  double R[9];
  double t[3];
} or_pose;

typedef struct {
  double fx, fy, cx, cy;
  int W, H;
} or_cam;

/* Per-surfel, per-camera state that the per-pixel evaluation reads. */
typedef struct {
  int visible;
  double pc[3];     /* surfel centre in the camera frame */
  double M[9];      /* row-major 3x3 with columns s_u t_u^c, s_v t_v^c, p_c (Eq. 1 in camera frame) */
  double opacity;
  double rc2;       /* (u,v) radius^2 of the support {o G >= 1/255}: 2 ln(255 o) */
  double lp2;       /* pixel radius^2 of the low-pass support: ln(255 o) */
  double cx, cy;    /* projected centre pi(p_c) (Eq. 3) */
  double rgb[3];
  float key;        /* the depth-order key: p_c.z in float32 arithmetic (or_depth_key) */
  double box[4];    /* xmin, xmax, ymin, ymax enclosing the whole support (a cheap exact reject) */
  int prim;         /* 0: surfel; 1: ellipsoid */
  double conic[3];  /* ellipsoid: inverse of the 2-D screen covariance (xx, xy, yy) */
  double su, sv;    /* surfel scales: the lengths of the columns s_u t_u^c, s_v t_v^c */
  double pscale;    /* |P| + |t|: the magnitude a float32 camera transform of the centre rounds */
} or_splat;

/* First-order bound on the float32 error of a surfel's rho3 at pixel (x, y),
 * whose FP64 value is rho3 at intersection depth lam (0 for ellipsoids). */
double or_rho3_err(const or_splat *s, const or_cam *cam, double x, double y, double rho3, double lam);

/* ---- constants of the blending rule (3DGS/2DGS rasterizer conventions) ---- */
#define OR_Z_NEAR 0.2
#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_ALPHA_MAX 0.99
#define OR_T_MIN 1e-4

/* Class bits of the affiliated-eye pixel map. */
#define OR_CLS_HOLE 1
#define OR_CLS_GAP 2
#define OR_CLS_CENTRE 4
#define OR_CLS_STRIP 8
#define OR_CLS_RENDER 16

int or_num_threads(void);

/* Sec. 3.3 / Eq. 1: unit-quaternion rotation; returns 0 for a zero quaternion. */
int or_quat_to_rot(const float q[4], double R[9]);
/* Real SH basis up to degree 3 evaluated at unit direction d; Y has (deg+1)^2 entries. */
void or_sh_basis(int deg, const double d[3], double *Y);

/* Per-surfel preparation for one camera (Sec. 3.3, Eq. 1-3). */
void or_prepare(const or_scene *sc, const or_pose *pose, const or_cam *cam, or_splat *out);

/* One ray-splat evaluation (Sec. 3.3, Eq. 2 and the ray-splat intersection).
 * Returns o*Ghat (before the 0.99 clamp); writes the contribution depth, rho3,
 * rho2 (both in the exponent's units). */
double or_eval(const or_splat *s, const or_cam *cam, double x, double y, double *depth,
               double *rho3, double *rho2);

/* Stage 1: full front-to-back render of the pixels in the window
 * [x0, x0+w) x [y0, y0+h), RGB and depth proxy D = sum d_i w_i from the same
 * weights w_i = alpha_i T_i. Outputs are w*h planar buffers for the window.
 * margin (optional) receives, per pixel, the smallest relative distance of a
 * decision that can move the result by more than 1e-5 to its threshold.
 * pairs (optional) receives the number of in-support evaluations.
 * fp32_bound (optional) receives, per pixel, a first-order bound on the error
 * of a float32 evaluation of the same blending sum (see render.c); with it
 * requested, the margins also take the float32 error of each surfel's rho3
 * (or_rho3_err) into account: a skip decision closer to its threshold than
 * that error gets a negative margin.
 * Returns the number of visible surfels, or -1 on bad arguments. */
int or_render(const or_scene *sc, const or_pose *pose, const or_cam *cam, const double bg[3],
              int x0, int y0, int w, int h, double *rgb, double *depth, double *trans,
              double *margin, int64_t *pairs, double *fp32_bound);

/* Render only the pixels whose tile (tile x tile) is set in tile_mask, writing
 * full-frame planar buffers (other pixels untouched). */
int or_render_tiles(const or_scene *sc, const or_pose *pose, const or_cam *cam, const double bg[3],
                    int tile, const uint8_t *tile_mask, double *rgb, double *depth, double *trans);

/* Integer tile rectangle of a surfel from (float) support bounds. rect = tx0, ty0,
 * tx1, ty1 inclusive; returns the tile count (0 if the bounds miss the image). */
int or_tile_rect(const float bounds[4], int W, int H, int tile, int rect[4]);

/* Every (surfel, tile) pair such that some pixel centre of the tile has
 * alpha >= 1/255 (the minimal binning of a tile rasterizer). Returns the count;
 * only the first cap pairs are written. */
int64_t or_support_pairs(const or_scene *sc, const or_pose *pose, const or_cam *cam, int tile, int64_t cap,
                         uint32_t *ids, uint32_t *tiles);

/* Whether the rectangle [x0,x1]x[y0,y1] meets the support of a surfel given as a
 * 12-float blend record (centre, log2 o, depth | 2x2 plane map | Az, Bz, Cz, _)
 * with squared radius k (FP64 evaluation of float inputs). */
int or_tile_test(const float rec[12], double k, double x0, double x1, double y0, double y1);

/* The depth-order key of a centre p (float32 scene position) for a pose. */
float or_depth_key(const or_pose *pose, const float p[3]);
/* Stable sort of (key, value) pairs by key (merge sort). */
void or_sort_pairs(int64_t n, uint64_t *keys, uint32_t *vals);

/* Stage 2 (Eq. 3-5): forward warp of the dominant image to the affiliated eye
 * with a depth test. Per source pixel: tgt = target linear index or -1, zkey =
 * float32 depth key (+inf for a background sample), tmargin = distance of the
 * target coordinate to a rounding boundary (+inf without a target). Per
 * destination pixel: winner = source linear index or -1 (hole), zdst = the
 * winner's key, out_rgb = the copied colour (0 at holes), hole = 1 at holes. */
void or_warp(const or_cam *cam, const or_pose *src, const or_pose *dst, const double *rgb,
             const double *D, const double *T, int64_t *tgt, float *zkey, double *tmargin,
             int64_t *winner, float *zdst, double *out_rgb, uint8_t *hole);

/* min/max of the alpha-normalised depth over valid pixels; returns the count. */
int64_t or_depth_range(int npix, const double *D, const double *T, double *dmin, double *dmax);

/* Step 1 (Eq. 6-8): edge ROI widths (left, right, top, bottom) and tile-aligned
 * strips strips[k] = x0, y0, x1, y1 (half-open pixels, x1 == x0 if absent).
 * margin = smallest distance of a sample to a rounding boundary. */
void or_edge_roi(const or_cam *cam, const or_pose *src, const or_pose *dst, int nsamples,
                 double dmin, double dmax, int m, int tile, int widths[4], int strips[16],
                 double *margin);

/* Stage 3/4: classification of holes outside the edge strips into gaps (filled by
 * linear interpolation) and centre holes. rgb_in/rgb_out planar [3][H][W]. */
void or_classify(int W, int H, const uint8_t *hole, const double *rgb_in, const uint8_t *in_strip,
                 int gap_thresh, int center_enabled, uint8_t *cls, double *rgb_out);

/* Step 2: 4-connected components of the centre-hole pixels (cls & OR_CLS_CENTRE),
 * bounding boxes expanded by m and aligned outward to tiles, in the order of each
 * component's smallest linear pixel index. rects[k] = x0, y0, x1, y1 half-open.
 * Returns the number of components (rects beyond cap are not written). */
int or_center_rois(int W, int H, const uint8_t *cls, int m, int tile, int *rects, int cap);

/* Whole stereo method with the oracle's own intermediates. All outputs are
 * full-frame; cls gets the class bits above; rects/nrects the centre ROIs. */
typedef struct {
  int gap_thresh, margin, nsamples, enable_center, depth_mode, tile;
  double dmin, dmax;
} or_params;

int or_stereo(const or_scene *sc, const or_pose *dom, const or_pose *aff, const or_cam *cam,
              const double bg[3], const or_params *p, double *rgb_dom, double *depth_dom,
              double *trans_dom, double *rgb_aff, uint8_t *cls, int widths[4], int *rects,
              int rect_cap, int *nrects, uint8_t *tile_mask);

#ifdef __cplusplus
}
#endif
#endif
