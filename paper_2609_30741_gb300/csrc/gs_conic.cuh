// The screen-space support of a surfel (or an ellipsoid, whose record has the
// same form), as the binning uses it: which tiles of a tile row the support can
// reach at a pixel centre. The support is grown by a float32 slack, so a pair
// it rules out never has alpha >= 1/255 in the rasterizer.
#pragma once

#include "gs_internal.cuh"

namespace gs {

// Screen-space conic of a surfel's 3D support. With d = x - c the homogeneous
// plane point is p = (d.x a + d.y b, d.x a' + d.y b', Az + d.x Bz + d.y Cz), so
// u = p.x/p.z, v = p.y/p.z and the support u^2 + v^2 <= k is
// Q(d) = p.x^2 + p.y^2 - k p.z^2 = d^T S d + 2 g.d + h <= 0, an ellipse that
// contains c. A tile is hit when the x-extent of the support inside the tile
// row's band meets the tile's pixel-centre columns; make_conic holds the
// quantities that give that x-extent in closed form. `ok` is false when the
// conic is not a well-conditioned ellipse in float32; callers then bin the whole
// bounding rectangle.
struct Conic {
  float Sxx, Sxy, Syy, gx, gy, h, dcx, dcy, ex, ey, rl2;
  float inv_sxx, slope;  // 1 / Sxx and Sxy / Syy
  bool ok;
};

// approximate square root and reciprocal (PTX); the 1e-3 slack of the support
// radius covers their error
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx_b(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ Conic make_conic(const float4 r0, const float4 r1, const float4 r2) {
  Conic q;
  const float k = fmaxf(r0.z, 0.f) * 1.001f + 1e-6f;  // r_c^2 grown by 1e-3
  const float ax = r1.x, ay = r1.y, az = r2.y, bx = r1.z, by = r1.w, bz = r2.z, A0 = r2.x;
  q.Sxx = fmaf(ax, ax, fmaf(ay, ay, -k * az * az));
  q.Syy = fmaf(bx, bx, fmaf(by, by, -k * bz * bz));
  q.Sxy = fmaf(ax, bx, fmaf(ay, by, -k * az * bz));
  q.gx = -k * A0 * az;
  q.gy = -k * A0 * bz;
  q.h = -k * A0 * A0;
  q.rl2 = 0.5f * k;
  const float det = fmaf(q.Sxx, q.Syy, -q.Sxy * q.Sxy);
  q.ok = q.Sxx > 0.f && q.Syy > 0.f && det > 1e-4f * q.Sxx * q.Syy;
  const float idet = q.ok ? rcp_approx_b(det) : 0.f;
  q.dcx = fmaf(q.Sxy, q.gy, -q.Syy * q.gx) * idet;
  q.dcy = fmaf(q.Sxy, q.gx, -q.Sxx * q.gy) * idet;
  const float Qc = fmaf(q.gx, q.dcx, fmaf(q.gy, q.dcy, q.h));
  q.ok = q.ok && Qc < 0.f;
  q.ex = q.ok ? sqrt_approx(-Qc * q.Syy * idet) * 1.0005f : 0.f;
  q.ey = q.ok ? sqrt_approx(-Qc * q.Sxx * idet) * 1.0005f : 0.f;
  q.inv_sxx = q.ok ? rcp_approx_b(q.Sxx) : 0.f;
  q.slope = q.ok ? q.Sxy * rcp_approx_b(q.Syy) : 0.f;
  return q;
}

// x-interval [lo, hi] (relative to c) of (ellipse u disc) within the band
// dy in [b0, b1]; the two parts are returned separately (empty: lo > hi).
__device__ __forceinline__ void band_slices(const Conic &q, float b0, float b1, float &elo, float &ehi, float &dlo,
                                            float &dhi) {
  elo = 3.0e38f;
  ehi = -3.0e38f;
  if (!(b1 < q.dcy - q.ey || b0 > q.dcy + q.ey)) {
    const float dyR = fmaf(-q.slope, q.ex, q.dcy), dyL = fmaf(q.slope, q.ex, q.dcy);
    if (dyR >= b0 && dyR <= b1) ehi = q.dcx + q.ex;  // rightmost point inside the band
    if (dyL >= b0 && dyL <= b1) elo = q.dcx - q.ex;  // leftmost point inside the band
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float y = e ? b1 : b0;
      if (y < q.dcy - q.ey || y > q.dcy + q.ey) continue;
      const float beta = fmaf(q.Sxy, y, q.gx);
      const float gamma = fmaf(fmaf(q.Syy, y, 2.f * q.gy), y, q.h);
      const float s = sqrt_approx(fmaxf(fmaf(beta, beta, -q.Sxx * gamma), 0.f));
      ehi = fmaxf(ehi, (s - beta) * q.inv_sxx);
      elo = fminf(elo, (-s - beta) * q.inv_sxx);
    }
    // grow by the same relative slack as the extents (float32 safety)
    const float pad = 5e-4f * q.ex + 1e-3f;
    elo -= pad;
    ehi += pad;
  }
  const float dyc = (b0 <= 0.f && b1 >= 0.f) ? 0.f : fminf(fabsf(b0), fabsf(b1));
  const float r2 = q.rl2 - dyc * dyc;
  if (r2 >= 0.f) {
    const float hw = sqrt_approx(r2);
    dlo = -hw;
    dhi = hw;
  } else {
    dlo = 3.0e38f;
    dhi = -3.0e38f;
  }
}

}  // namespace gs
