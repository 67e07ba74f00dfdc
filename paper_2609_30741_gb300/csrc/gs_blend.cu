// Per-tile front-to-back alpha blending with the joint depth proxy.
//
// Paper: Sec. 3.1 Stage 1 - every contributing surfel gets the weight
// w_i = alpha_i T_i, and the same weight accumulates the colour C = sum c_i w_i
// and the depth proxy D = sum d_i w_i in one pass (no separate depth pass).
// Sec. 3.3 (Eq. 2 and the ray-splat intersection) gives alpha.
//
// One CTA of 64 threads renders one 16x16 tile; every thread blends four pixels
// of one column, 4 rows apart. The homogeneous plane point p of a pixel is
// affine in the pixel position, so the thread evaluates p once and steps it by
// 4 rows with three additions; each surfel record read from shared memory
// serves four evaluations. The tile's depth-sorted surfel ids are consumed in
// batches of 128 whose 64-byte records are staged in shared memory (structure
// of arrays: one broadcast float4 per field); cp.async double-buffers the next
// batch behind the current one. A CTA leaves as soon as all 256 pixels have
// terminated (__syncthreads_count).
#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int kBatch = 128;          // records per stage: 2 x 128 x 64 B = 16 KB of shared memory
constexpr int kBlendThreads = 64;    // 16 columns x 4 row groups
constexpr int kPix = 4;              // pixels per thread, kRowStep rows apart
constexpr int kRowStep = 4;
// 1 / (2 ln 2): log2(o Ghat) = (r_c^2 - rho) / (2 ln 2) + log2(1/255)
constexpr float kHalfLog2e = 0.72134752044448170f;

template <bool MASKED, bool STATS, bool COUNT>
__global__ void __launch_bounds__(kBlendThreads) blend_kernel(const uint2 *__restrict__ ranges,
                                                              const uint32_t *__restrict__ ids,
                                                              const float4 *__restrict__ rec,
                                                              const CamBlock *__restrict__ cams, int eye,
                                                              const uint8_t *__restrict__ mask, float3 bg,
                                                              float *__restrict__ rgb, float *__restrict__ depth,
                                                              float *__restrict__ trans, uint8_t *__restrict__ cls,
                                                              Counters *__restrict__ ctr, uint32_t n_rec) {
  const int tile = blockIdx.x;
  if (MASKED && !mask[tile]) return;
  const int W = cams->eye[eye].W, H = cams->eye[eye].H, tiles_x = cams->eye[eye].tiles_x;
  const int px = (tile % tiles_x) * kTile + (threadIdx.x & 15);
  const int py = (tile / tiles_x) * kTile + (threadIdx.x >> 4);  // first of rows py, py + 4, py + 8, py + 12
  const uint2 rg = ranges[tile];

  __shared__ float4 s0[2][kBatch], s1[2][kBatch], s2[2][kBatch], s3[2][kBatch];

  const float fx = (float)px, fy = (float)py;
  float T[kPix], C0[kPix], C1[kPix], C2[kPix], D[kPix];
  unsigned live = 0;  // bit k: pixel k still blending
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    T[k] = 1.f; C0[k] = C1[k] = C2[k] = D[k] = 0.f;
    if (px < W && py + kRowStep * k < H) live |= 1u << k;
  }
  unsigned npairs = 0, ncontrib = 0;

  auto stage = [&](int buf, uint32_t b0) {
#pragma unroll
    for (int h = 0; h < kBatch / kBlendThreads; ++h) {
      const int slot = threadIdx.x + h * kBlendThreads;
      const uint32_t i = b0 + (uint32_t)slot;
      if (i < rg.y) {
        const uint32_t id = ids[i];
        if (id < n_rec) {
          const float4 *r = rec + 4 * (size_t)id;
          cp_async16(&s0[buf][slot], r + 0);
          cp_async16(&s1[buf][slot], r + 1);
          cp_async16(&s2[buf][slot], r + 2);
          cp_async16(&s3[buf][slot], r + 3);
        } else {  // never expected; a record that cannot contribute keeps reads in bounds
          s0[buf][slot] = make_float4(0.f, 0.f, -1.f, 1.f);
          s1[buf][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
          s2[buf][slot] = make_float4(1.f, 0.f, 0.f, 0.f);
          s3[buf][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
    cp_async_commit();
  };

  int buf = 0;
  if (rg.x < rg.y) stage(0, rg.x);
  for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBatch, buf ^= 1) {
    cp_async_wait_all();
    // barrier: the batch in `buf` is visible to all, and every thread has
    // finished reading the other buffer, which the prefetch below overwrites
    if (__syncthreads_count(live == 0u) == kBlendThreads) break;
    if (b0 + kBatch < rg.y) stage(buf ^ 1, b0 + kBatch);
    const int nb = (int)min((uint32_t)kBatch, rg.y - b0);
    for (int j = 0; j < nb && live; ++j) {
      const float4 a = s0[buf][j];
      const float4 b = s1[buf][j];
      const float4 c = s2[buf][j];
      // homogeneous plane point at the thread's first pixel and its 4-row step
      const float dx = fx - a.x, dy = fy - a.y;
      float qx = fmaf(dx, b.x, dy * b.z);
      float qy = fmaf(dx, b.y, dy * b.w);
      float qz = fmaf(dy, c.z, fmaf(dx, c.y, c.x));
      const float sx = kRowStep * b.z, sy = kRowStep * b.w, sz = kRowStep * c.z;
      const float dx2 = dx * dx;
      float dyk = dy;
#pragma unroll
      for (int k = 0; k < kPix; ++k) {
        if (live & (1u << k)) {
          const float iq = rcp_approx(qz);
          const float u = qx * iq, v = qy * iq;
          const float rho3 = fmaf(u, u, v * v);
          const float h = fmaf(dyk, dyk, dx2);
          const float rho2 = h + h;  // low-pass term 2 |x - c|^2, same exponent units
          const float rho = fminf(rho3, rho2);
          if (COUNT) ++npairs;
          if (rho <= a.z) {  // alpha >= 1/255
            const float alpha = fminf(kAlphaMax, ex2_approx(fmaf(a.z - rho, kHalfLog2e, kLog2AlphaMin)));
            const float Tn = fmaf(-T[k], alpha, T[k]);
            if (Tn < kTMin) {
              live &= ~(1u << k);
            } else {
              const float4 d = s3[buf][j];
              const float z = rho3 <= rho2 ? fmaf(c.w, u, fmaf(d.x, v, a.w)) : a.w;
              const float w = alpha * T[k];
              if (COUNT) ++ncontrib;
              C0[k] = fmaf(w, d.y, C0[k]);
              C1[k] = fmaf(w, d.z, C1[k]);
              C2[k] = fmaf(w, d.w, C2[k]);
              D[k] = fmaf(w, z, D[k]);
              T[k] = Tn;
            }
          }
        }
        qx += sx;
        qy += sy;
        qz += sz;
        dyk += (float)kRowStep;
      }
    }
  }
  cp_async_wait_all();

  const size_t hw = (size_t)W * H;
  float lo = 3.0e38f, hi = 0.f;
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    const int y = py + kRowStep * k;
    if (px >= W || y >= H) continue;
    const size_t p = (size_t)y * W + px;
    rgb[p] = fmaf(T[k], bg.x, C0[k]);
    rgb[hw + p] = fmaf(T[k], bg.y, C1[k]);
    rgb[2 * hw + p] = fmaf(T[k], bg.z, C2[k]);
    if (depth) depth[p] = D[k];
    if (trans) trans[p] = T[k];
    if (MASKED && cls) cls[p] |= (uint8_t)kClsRender;
    if (STATS && 1.f - T[k] >= 0.5f) {
      // range of the alpha-normalised depth D / (1 - T) over pixels with coverage >= 0.5
      const float dh = D[k] / (1.f - T[k]);
      lo = fminf(lo, dh);
      hi = fmaxf(hi, dh);
    }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0 && hi > 0.f) {
      atomicMin(&ctr->dmin_bits, __float_as_uint(fmaxf(lo, 0.f)));
      atomicMax(&ctr->dmax_bits, __float_as_uint(hi));
    }
  }
  if (COUNT) {
    unsigned long long v = npairs, cc = ncontrib;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, o);
      cc += __shfl_xor_sync(0xffffffffu, cc, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&ctr->pairs[eye], v);
      atomicAdd(&ctr->contrib[eye], cc);
    }
  }
}

template <bool M, bool S, bool C>
static void launch_variant(int ntiles, cudaStream_t s, const Workspace &ws, const uint32_t *ids, int eye,
                           const uint8_t *mask, float3 bg, float *rgb, float *depth, float *trans, uint8_t *cls) {
  blend_kernel<M, S, C><<<ntiles, kBlendThreads, 0, s>>>(ws.ranges, ids, ws.rec[eye], ws.cams, eye, mask, bg, rgb,
                                                         depth, trans, cls, ws.ctr, (uint32_t)ws.max_surfels);
  GS_LAUNCHED(1);
}

cudaError_t launch_blend(const Workspace &ws, int eye, int W, int H, const uint8_t *tile_mask, float3 bg, float *rgb,
                         float *depth, float *trans, uint8_t *cls, bool depth_stats, bool count_pairs,
                         cudaStream_t s) {
  const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile, ntiles = tx * ty;
  if (ntiles == 0) return cudaSuccess;
  const uint32_t *ids = ws.ival;
  const bool m = tile_mask != nullptr;
#define GS_BLEND(M, S, C) launch_variant<M, S, C>(ntiles, s, ws, ids, eye, tile_mask, bg, rgb, depth, trans, cls)
  if (m) {
    if (count_pairs) GS_BLEND(true, false, true); else GS_BLEND(true, false, false);
  } else if (depth_stats) {
    if (count_pairs) GS_BLEND(false, true, true); else GS_BLEND(false, true, false);
  } else {
    if (count_pairs) GS_BLEND(false, false, true); else GS_BLEND(false, false, false);
  }
#undef GS_BLEND
  return cudaGetLastError();
}

}  // namespace gs
