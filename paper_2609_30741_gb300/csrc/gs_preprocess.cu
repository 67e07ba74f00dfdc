// Camera set-up (FP64) and per-surfel preprocessing for one or both eyes.
//
// Paper: Sec. 3.3 (2D Gaussian surfels, Eq. 1-2, ray-splat intersection),
// Sec. 3.4 (pinhole projection, Eq. 3; poses, Eq. 4-5), Sec. 3.1 Stage 1;
// Sec. 3.2 (the pipeline accepts any Gaussian splatting variant with per-pixel
// depth: the 3D ellipsoids of 3DGS are prepared below as well).
#include "gs_internal.cuh"
#include "gs_launch.cuh"

namespace gs {

// ---------------------------------------------------------------- FP64 set-up
//
// The only double-precision work on the GPU: inverting the camera-to-world
// poses (world -> camera) and composing the relative pose between the eyes,
// X_aff = R_aff^T R_dom X_dom + R_aff^T (t_dom - t_aff) (Eq. 4 followed by Eq. 5).
__global__ void setup_cams_kernel(PoseArgs pa, CamBlock *cams) {
  griddep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  CamBlock cb;
  for (int e = 0; e < 2; ++e) {
    const int src = e < pa.neyes ? e : 0;
    const double *R = pa.R[src], *t = pa.t[src];
    EyeCam &c = cb.eye[e];
    for (int i = 0; i < 3; ++i) {
      double ti = 0.0;
      for (int j = 0; j < 3; ++j) {
        c.R[i * 3 + j] = (float)R[j * 3 + i];  // transpose
        ti -= R[j * 3 + i] * t[j];
      }
      c.t[i] = (float)ti;
      c.centre[i] = (float)t[i];
    }
    c.fx = (float)pa.fx; c.fy = (float)pa.fy; c.cx = (float)pa.cx; c.cy = (float)pa.cy;
    c.W = pa.W; c.H = pa.H;
    c.tshift = e == 0 ? pa.tshift : pa.tshift1;
    c.tiles_x = (pa.W + (1 << c.tshift) - 1) >> c.tshift;
    c.tiles_y = (pa.H + (1 << c.tshift) - 1) >> c.tshift;
  }
  // A parallel rig (equal orientation, baseline in the image plane, Sec. 4.2):
  // both cameras measure the same depth, z_aff = z_dom in exact arithmetic. The
  // two offsets differ only by FP64 rounding of R^T R = I, so the affiliated eye
  // takes the dominant one and both eyes' depth keys are bit-identical.
  if (pa.parallel) cb.eye[1].t[2] = cb.eye[0].t[2];
  const int a = pa.neyes > 1 ? 1 : 0;
  const double *Rd = pa.R[0], *td = pa.t[0], *Ra = pa.R[a], *ta = pa.t[a];
  for (int i = 0; i < 3; ++i) {
    double tr = 0.0;
    for (int j = 0; j < 3; ++j) {
      double r = 0.0;
      for (int k = 0; k < 3; ++k) r += Ra[k * 3 + i] * Rd[k * 3 + j];
      cb.Rrel[i * 3 + j] = (float)r;
      tr += Ra[j * 3 + i] * (td[j] - ta[j]);
    }
    cb.trel[i] = (float)tr;
  }
  *cams = cb;
}

const void *setup_cams_kernel_ptr() { return (const void *)setup_cams_kernel; }

cudaError_t launch_setup_cams(const PoseArgs &pa, CamBlock *cams, cudaStream_t s) {
  launch_k(setup_cams_kernel, 1, 32, 0, s, pa, cams);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- SH colour
//
// Real spherical harmonics up to degree 3 (3DGS sign convention). Constants are
// the closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times each polynomial's
// normalisation, written out to float precision.
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float b[16]) {
  const float Y00 = 0.28209479177387814f;        // 1 / (2 sqrt(pi))
  const float Y1 = 0.48860251190291992f;         // sqrt(3 / (4 pi))
  const float Y2a = 1.0925484305920792f;         // sqrt(15 / pi) / 2
  const float Y2b = 0.31539156525252001f;        // sqrt(5 / pi) / 4
  const float Y2c = 0.54627421529603959f;        // sqrt(15 / pi) / 4
  const float Y3a = 0.59004358992664352f;        // sqrt(35 / (2 pi)) / 4
  const float Y3b = 2.8906114426405538f;         // sqrt(105 / pi) / 2
  const float Y3c = 0.45704579946446572f;        // sqrt(21 / (2 pi)) / 4
  const float Y3d = 0.37317633259011540f;        // sqrt(7 / pi) / 4
  const float Y3e = 1.4453057213202769f;         // sqrt(105 / pi) / 4
  b[0] = Y00;
  if (DEG >= 1) {
    b[1] = -Y1 * y; b[2] = Y1 * z; b[3] = -Y1 * x;
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    b[4] = Y2a * x * y; b[5] = -Y2a * y * z; b[6] = Y2b * (2.f * zz - xx - yy);
    b[7] = -Y2a * x * z; b[8] = Y2c * (xx - yy);
    if (DEG >= 3) {
      b[9] = -Y3a * y * (3.f * xx - yy);
      b[10] = Y3b * x * y * z;
      b[11] = -Y3c * y * (4.f * zz - xx - yy);
      b[12] = Y3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      b[13] = -Y3c * x * (4.f * zz - xx - yy);
      b[14] = Y3e * z * (xx - yy);
      b[15] = -Y3a * x * (xx - 3.f * yy);
    }
  }
}

// Both eyes' colours of primitive i centred at p: max(0, 0.5 + sum_k Y_k(dir)
// c_k) with dir the unit vector from the eye's centre to p. The coefficients
// are streamed once from memory (float4 loads at degree 3, whose 48 floats per
// primitive keep the alignment the scene check demands) and every index is a
// compile-time constant, so
// nothing goes through local memory; each channel's sum runs in the order k = 0,
// 1, ... for both eyes.
template <int DEG>
__device__ __forceinline__ void sh_colours(const gs_scene &sc, int i, bool load, const CamBlock *cams, int neyes,
                                           float4 p, float rgb[2][3]) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  float b[2][16];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const EyeCam &c = cams->eye[e < neyes ? e : 0];
    const float dx = p.x - c.centre[0], dy = p.y - c.centre[1], dz = p.z - c.centre[2];
    const float dn = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    sh_basis<DEG>(dx * dn, dy * dn, dz * dn, b[e]);
  }
  float acc[2][3] = {{0.5f, 0.5f, 0.5f}, {0.5f, 0.5f, 0.5f}};
  const float *src = sc.sh + (size_t)i * K * 3;
  if (load) {
    if (DEG == 3) {  // 48 floats: the scene's SH array is 16-byte aligned at degree 3
      const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
      for (int m = 0; m < 3 * K / 4; ++m) {
        const float4 v = s4[m];
        const float cf[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = 4 * m + u;
#pragma unroll
          for (int e = 0; e < 2; ++e) acc[e][j % 3] = fmaf(b[e][j / 3], cf[u], acc[e][j % 3]);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 3 * K; ++j) {
        const float cf = src[j];
#pragma unroll
        for (int e = 0; e < 2; ++e) acc[e][j % 3] = fmaf(b[e][j / 3], cf, acc[e][j % 3]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) rgb[e][ch] = fmaxf(acc[e][ch], 0.f);
}

// Tile rectangle of the pixels whose centres lie inside [xmin, xmax] x
// [ymin, ymax]; the count is 0 when none does.
__device__ __forceinline__ uint32_t tile_rect(const EyeCam &c, float xmin, float xmax, float ymin, float ymax,
                                              ushort4 &rect) {
  rect = make_ushort4(0, 0, 0, 0);
  if (!(xmax >= 0.f && ymax >= 0.f && xmin <= c.W - 1.f && ymin <= c.H - 1.f)) return 0;
  const int px0 = xmin <= 0.f ? 0 : (int)ceilf(xmin);
  const int px1 = xmax >= c.W - 1.f ? c.W - 1 : (int)floorf(xmax);
  const int py0 = ymin <= 0.f ? 0 : (int)ceilf(ymin);
  const int py1 = ymax >= c.H - 1.f ? c.H - 1 : (int)floorf(ymax);
  if (px0 > px1 || py0 > py1) return 0;
  rect = make_ushort4(px0 >> c.tshift, py0 >> c.tshift, px1 >> c.tshift, py1 >> c.tshift);
  return (uint32_t)(rect.z - rect.x + 1) * (uint32_t)(rect.w - rect.y + 1);
}

// ---------------------------------------------------------------- preprocess
//
// One thread per surfel; the attributes are read once (coalesced float4 loads)
// and both eyes are prepared from registers.
//
// Blend record. With M = [s_u t_u^c, s_v t_v^c, p_c] (Eq. 1 in the camera frame)
// the pixel ray through (x, y) meets the surfel plane at the local (u, v) with
// (u, v, 1) ~ (T_u - x T_w) x (T_v - y T_w) where T = K M (the 2DGS plane
// intersection). Writing x = c_x + dx, y = c_y + dy around the projected centre c
// and dividing by p_c.z > 0 gives the affine form
//   p.x = dx V1 - dy U1,   p.y = -dx V0 + dy U0,   p.z = Az + dx Bz + dy Cz
// with U = fx (M_row0 - (p_x/p_z) M_row2), V = fy (M_row1 - (p_y/p_z) M_row2)
// (both zero in the third column), Az = (U0 V1 - U1 V0)/p_z,
// Bz = (V0 M21 - V1 M20)/p_z, Cz = (M20 U1 - M21 U0)/p_z, so u = p.x/p.z,
// v = p.y/p.z. Expanding around c keeps the terms small (well conditioned).
// The intersection depth is z = M20 u + M21 v + p_z.
template <int DEG>
__global__ void __launch_bounds__(256) preprocess_kernel(gs_scene sc, const CamBlock *__restrict__ cams,
                                                         Workspace ws, int neyes) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.n) return;
  const float4 p4 = reinterpret_cast<const float4 *>(sc.pos)[i];
  float4 q = reinterpret_cast<const float4 *>(sc.quat)[i];
  const float2 s2 = reinterpret_cast<const float2 *>(sc.scale)[i];
  const float o = sc.opacity[i];
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  bool alive = qn2 > 0.f && 255.f * o >= 1.f;
  // normalise (w, x, y, z) and build the two tangent columns of R (Eq. 1)
  const float qi = alive ? rsqrtf(qn2) : 0.f;
  const float w = q.x * qi, x = q.y * qi, y = q.z * qi, z = q.w * qi;
  const float tu[3] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y)};
  const float tv[3] = {2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x)};
  // support radius in (u, v): o G >= 1/255  <=>  u^2 + v^2 <= 2 ln(255 o)
  const float rc2 = alive ? 2.f * logf(255.f * o) : 0.f;
  const float rc = sqrtf(fmaxf(rc2, 0.f));
  const float lp = sqrtf(fmaxf(0.5f * rc2, 0.f));  // low-pass support radius, pixels
  float rgbs[2][3];
  sh_colours<DEG>(sc, i, alive, cams, neyes, p4, rgbs);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (e >= neyes) break;
    const EyeCam &c = cams->eye[e];
    bool vis = alive;
    float pc[3], tuc[3], tvc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      pc[r] = fmaf(c.R[r * 3 + 0], p4.x, fmaf(c.R[r * 3 + 1], p4.y, fmaf(c.R[r * 3 + 2], p4.z, c.t[r])));
      tuc[r] = fmaf(c.R[r * 3 + 0], tu[0], fmaf(c.R[r * 3 + 1], tu[1], c.R[r * 3 + 2] * tu[2]));
      tvc[r] = fmaf(c.R[r * 3 + 0], tv[0], fmaf(c.R[r * 3 + 1], tv[1], c.R[r * 3 + 2] * tv[2]));
    }
    vis = vis && pc[2] > kZNear;
    const float M0[3] = {s2.x * tuc[0], s2.y * tvc[0], pc[0]};
    const float M1[3] = {s2.x * tuc[1], s2.y * tvc[1], pc[1]};
    const float M2[3] = {s2.x * tuc[2], s2.y * tvc[2], pc[2]};
    // screen bounds: the four projected corners of the support square plus the
    // low-pass disc around the projected centre
    float xmin = 3.0e38f, xmax = -3.0e38f, ymin = 3.0e38f, ymax = -3.0e38f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float a = (k & 1) ? rc : -rc, b = (k & 2) ? rc : -rc;
      const float X = fmaf(a, M0[0], fmaf(b, M0[1], pc[0]));
      const float Y = fmaf(a, M1[0], fmaf(b, M1[1], pc[1]));
      const float Z = fmaf(a, M2[0], fmaf(b, M2[1], pc[2]));
      vis = vis && Z > kZNear;
      const float iz = 1.f / fmaxf(Z, kZNear);
      const float u = fmaf(c.fx * X, iz, c.cx), v = fmaf(c.fy * Y, iz, c.cy);
      xmin = fminf(xmin, u); xmax = fmaxf(xmax, u);
      ymin = fminf(ymin, v); ymax = fmaxf(ymax, v);
    }
    const float izc = 1.f / fmaxf(pc[2], kZNear);
    const float rx = pc[0] * izc, ry = pc[1] * izc;
    const float cxp = fmaf(c.fx, rx, c.cx), cyp = fmaf(c.fy, ry, c.cy);
    xmin = fminf(xmin, cxp - lp) - kBoundPad; xmax = fmaxf(xmax, cxp + lp) + kBoundPad;
    ymin = fminf(ymin, cyp - lp) - kBoundPad; ymax = fmaxf(ymax, cyp + lp) + kBoundPad;
    // tile rectangle of the pixels whose centres lie inside the bounds
    ushort4 rect;
    uint32_t count = tile_rect(c, xmin, xmax, ymin, ymax, rect);
    if (!vis) {
      count = 0;
      rect = make_ushort4(0, 0, 0, 0);
    }
    ws.cnt[e][i] = count;
    ws.rect[e][i] = rect;
    ws.zkey[e][i] = __float_as_uint(pc[2]);
    ws.bounds[e][i] = make_float4(xmin, xmax, ymin, ymax);
    if (count == 0) continue;
    const float U0 = c.fx * fmaf(-rx, M2[0], M0[0]), U1 = c.fx * fmaf(-rx, M2[1], M0[1]);
    const float V0 = c.fy * fmaf(-ry, M2[0], M1[0]), V1 = c.fy * fmaf(-ry, M2[1], M1[1]);
    const float Az = fmaf(U0, V1, -U1 * V0) * izc;
    const float Bz = fmaf(V0, M2[1], -V1 * M2[0]) * izc;
    const float Cz = fmaf(M2[0], U1, -M2[1] * U0) * izc;
    // view-dependent colour from this eye's centre
    const float *rgb = rgbs[e];
    float4 *r = ws.rec[e] + 4 * (size_t)i;
    r[0] = make_float4(cxp, cyp, rc2, pc[2]);
    r[1] = make_float4(V1, -V0, -U1, U0);
    r[2] = make_float4(Az, Bz, Cz, M2[0]);
    r[3] = make_float4(M2[1], rgb[0], rgb[1], rgb[2]);
  }
}

// Ellipsoids (3DGS backbone), EWA splatting. With the camera-frame axes
// m_k = s_k W r_k (r_k the columns of Rq) the camera covariance is
// sum_k m_k m_k^T, and with j_k = J m_k the screen covariance is
// Sigma2D = sum_k j_k j_k^T + 0.3 I. Its determinant is assembled from
// non-negative terms (Cauchy-Binet plus the dilation), so it keeps its relative
// accuracy for elongated splats:
//   det = sum_{k<l} (j_k x j_l)^2 + 0.3 (|j_0|^2 + |j_1|^2 + |j_2|^2) + 0.09.
// The conic Q = Sigma2D^-1 = [[A, B], [B, C]] is stored as its upper Cholesky
// factor L = [[l00, l01], [0, l11]], Q = L^T L, in closed form:
// l00 = sqrt(cyy / det), l01 = -cxy / sqrt(det cyy), l11 = 1 / sqrt(cyy). The
// record keeps the surfel layout: r1 = (l00, 0, l01, l11) for the plane point's
// (x, y) rows, r2 = (1, 0, 0, 0) for a constant third coordinate and zero depth
// slopes, so the rasterizer's u^2 + v^2 is d^T Q d and its depth the centre's.
// The support d^T Q d <= 2 ln(255 o) has the half extents sqrt(k cxx) and
// sqrt(k cyy).
template <int DEG>
__global__ void __launch_bounds__(256) preprocess_ellipsoid_kernel(gs_scene sc, const CamBlock *__restrict__ cams,
                                                                   Workspace ws, int neyes) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.n) return;
  const float4 p4 = reinterpret_cast<const float4 *>(sc.pos)[i];
  const float4 q = reinterpret_cast<const float4 *>(sc.quat)[i];
  const float4 s4 = reinterpret_cast<const float4 *>(sc.scale)[i];
  const float o = sc.opacity[i];
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  const bool alive = qn2 > 0.f && 255.f * o >= 1.f;
  const float qi = alive ? rsqrtf(qn2) : 0.f;
  const float w = q.x * qi, x = q.y * qi, y = q.z * qi, z = q.w * qi;
  // the three columns of Rq, scaled by the axis lengths
  const float ax[3][3] = {
      {s4.x * (1.f - 2.f * (y * y + z * z)), s4.x * 2.f * (x * y + w * z), s4.x * 2.f * (x * z - w * y)},
      {s4.y * 2.f * (x * y - w * z), s4.y * (1.f - 2.f * (x * x + z * z)), s4.y * 2.f * (y * z + w * x)},
      {s4.z * 2.f * (x * z + w * y), s4.z * 2.f * (y * z - w * x), s4.z * (1.f - 2.f * (x * x + y * y))}};
  const float rc2 = alive ? 2.f * logf(255.f * o) : 0.f;
  float rgbs[2][3];
  sh_colours<DEG>(sc, i, alive, cams, neyes, p4, rgbs);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (e >= neyes) break;
    const EyeCam &c = cams->eye[e];
    float pc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      pc[r] = fmaf(c.R[r * 3 + 0], p4.x, fmaf(c.R[r * 3 + 1], p4.y, fmaf(c.R[r * 3 + 2], p4.z, c.t[r])));
    const bool vis = alive && pc[2] > kZNear;
    const float izc = 1.f / fmaxf(pc[2], kZNear);
    const float rx = pc[0] * izc, ry = pc[1] * izc;
    const float gx = c.fx * izc, gy = c.fy * izc;
    float jx[3], jy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float mx = fmaf(c.R[0], ax[k][0], fmaf(c.R[1], ax[k][1], c.R[2] * ax[k][2]));
      const float my = fmaf(c.R[3], ax[k][0], fmaf(c.R[4], ax[k][1], c.R[5] * ax[k][2]));
      const float mz = fmaf(c.R[6], ax[k][0], fmaf(c.R[7], ax[k][1], c.R[8] * ax[k][2]));
      jx[k] = gx * fmaf(-rx, mz, mx);
      jy[k] = gy * fmaf(-ry, mz, my);
    }
    const float txx = fmaf(jx[0], jx[0], fmaf(jx[1], jx[1], jx[2] * jx[2]));
    const float tyy = fmaf(jy[0], jy[0], fmaf(jy[1], jy[1], jy[2] * jy[2]));
    const float cxy = fmaf(jx[0], jy[0], fmaf(jx[1], jy[1], jx[2] * jy[2]));
    const float cxx = txx + 0.3f, cyy = tyy + 0.3f;
    const float k01 = fmaf(jx[0], jy[1], -jy[0] * jx[1]);
    const float k02 = fmaf(jx[0], jy[2], -jy[0] * jx[2]);
    const float k12 = fmaf(jx[1], jy[2], -jy[1] * jx[2]);
    const float det = fmaf(k01, k01, fmaf(k02, k02, fmaf(k12, k12, fmaf(0.3f, txx + tyy, 0.09f))));
    const float cxp = fmaf(c.fx, rx, c.cx), cyp = fmaf(c.fy, ry, c.cy);
    const float ex = sqrtf(rc2 * cxx), ey = sqrtf(rc2 * cyy);
    const float xmin = cxp - ex - kBoundPad, xmax = cxp + ex + kBoundPad;
    const float ymin = cyp - ey - kBoundPad, ymax = cyp + ey + kBoundPad;
    ushort4 rect;
    uint32_t count = tile_rect(c, xmin, xmax, ymin, ymax, rect);
    if (!vis) {
      count = 0;
      rect = make_ushort4(0, 0, 0, 0);
    }
    ws.cnt[e][i] = count;
    ws.rect[e][i] = rect;
    ws.zkey[e][i] = __float_as_uint(pc[2]);
    ws.bounds[e][i] = make_float4(xmin, xmax, ymin, ymax);
    if (count == 0) continue;
    const float l00 = sqrtf(cyy / det);
    const float l01 = -cxy / sqrtf(det * cyy);
    const float l11 = rsqrtf(cyy);
    const float *rgb = rgbs[e];
    float4 *r = ws.rec[e] + 4 * (size_t)i;
    r[0] = make_float4(cxp, cyp, rc2, pc[2]);
    r[1] = make_float4(l00, 0.f, l01, l11);
    r[2] = make_float4(1.f, 0.f, 0.f, 0.f);
    r[3] = make_float4(0.f, rgb[0], rgb[1], rgb[2]);
  }
}

cudaError_t launch_preprocess(const gs_scene &sc, Workspace &ws, int neyes, int W, int H, cudaStream_t s) {
  (void)W; (void)H;
  ws.prim = sc.primitive;
  if (sc.n == 0) return cudaSuccess;
  const int g = (sc.n + 255) / 256;
  switch (sc.sh_degree + 4 * (sc.primitive == 1)) {
    case 0: launch_k(preprocess_kernel<0>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    case 1: launch_k(preprocess_kernel<1>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    case 2: launch_k(preprocess_kernel<2>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    case 3: launch_k(preprocess_kernel<3>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    case 4: launch_k(preprocess_ellipsoid_kernel<0>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    case 5: launch_k(preprocess_ellipsoid_kernel<1>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    case 6: launch_k(preprocess_ellipsoid_kernel<2>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
    default: launch_k(preprocess_ellipsoid_kernel<3>, g, 256, 0, s, sc, ws.cams, ws, neyes); break;
  }
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace gs
