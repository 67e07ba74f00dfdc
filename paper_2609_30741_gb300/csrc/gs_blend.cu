// Per-tile front-to-back alpha blending with the joint depth proxy.
//
// Paper: Sec. 3.1 Stage 1 - every contributing surfel gets the weight
// w_i = alpha_i T_i, and the same weight accumulates the colour C = sum c_i w_i
// and the depth proxy D = sum d_i w_i in one pass (no separate depth pass).
// Sec. 3.3 (Eq. 2 and the ray-splat intersection) gives alpha.
//
// One CTA renders one 16x16 tile, one thread per pixel. The tile's depth-sorted
// surfel ids are consumed in batches of 256 whose 64-byte records are staged in
// shared memory (structure of arrays, so every thread reads one broadcast
// float4 per field); cp.async double-buffers the next batch behind the current
// one. A CTA leaves as soon as every pixel has terminated (__syncthreads_count).
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

constexpr int kBatch = 256;

template <bool MASKED, bool STATS, bool COUNT>
__global__ void __launch_bounds__(256) blend_kernel(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ ids,
                                                    const float4 *__restrict__ rec, const CamBlock *__restrict__ cams,
                                                    int eye, const uint8_t *__restrict__ mask, float3 bg,
                                                    float *__restrict__ rgb, float *__restrict__ depth,
                                                    float *__restrict__ trans, uint8_t *__restrict__ cls,
                                                    Counters *__restrict__ ctr) {
  const int tile = blockIdx.x;
  if (MASKED && !mask[tile]) return;
  const int W = cams->eye[eye].W, H = cams->eye[eye].H, tiles_x = cams->eye[eye].tiles_x;
  const int px = (tile % tiles_x) * kTile + (threadIdx.x & 15);
  const int py = (tile / tiles_x) * kTile + (threadIdx.x >> 4);
  const bool inside = px < W && py < H;
  const uint2 rg = ranges[tile];

  __shared__ float4 s0[2][kBatch], s1[2][kBatch], s2[2][kBatch], s3[2][kBatch];

  const float fx = (float)px, fy = (float)py;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  bool done = !inside;
  unsigned npairs = 0, ncontrib = 0;

  auto stage = [&](int buf, uint32_t b0) {
    const uint32_t i = b0 + threadIdx.x;
    if (i < rg.y) {
      const float4 *r = rec + 4 * (size_t)ids[i];
      cp_async16(&s0[buf][threadIdx.x], r + 0);
      cp_async16(&s1[buf][threadIdx.x], r + 1);
      cp_async16(&s2[buf][threadIdx.x], r + 2);
      cp_async16(&s3[buf][threadIdx.x], r + 3);
    }
    cp_async_commit();
  };

  int buf = 0;
  if (rg.x < rg.y) stage(0, rg.x);
  for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBatch, buf ^= 1) {
    cp_async_wait_all();
    // barrier: the batch in `buf` is visible to all, and every thread has
    // finished reading the other buffer, which the prefetch below overwrites
    if (__syncthreads_count(done) == kBatch) break;
    if (b0 + kBatch < rg.y) stage(buf ^ 1, b0 + kBatch);
    const int nb = (int)min((uint32_t)kBatch, rg.y - b0);
    if (!done) {
      for (int j = 0; j < nb; ++j) {
        const float4 a = s0[buf][j];
        const float dx = fx - a.x, dy = fy - a.y;
        const float4 b = s1[buf][j];
        const float4 c = s2[buf][j];
        // homogeneous plane intersection (u, v, 1) ~ p (see preprocess)
        const float qx = fmaf(dx, b.x, dy * b.z);
        const float qy = fmaf(dx, b.y, dy * b.w);
        const float qz = fmaf(dy, c.z, fmaf(dx, c.y, c.x));
        const float iq = rcp_approx(qz);
        const float u = qx * iq, v = qy * iq;
        const float rho3 = fmaf(u, u, v * v);
        const float rho2 = 2.f * fmaf(dx, dx, dy * dy);  // low-pass term, same exponent units
        const float rho = fminf(rho3, rho2);
        const float lg = fmaf(rho, kNegHalfLog2e, a.z);  // log2(o * Ghat)
        if (COUNT) ++npairs;
        if (lg < kLog2AlphaMin) continue;  // alpha < 1/255
        const float alpha = fminf(kAlphaMax, ex2_approx(lg));
        const float Tn = fmaf(-T, alpha, T);
        if (Tn < kTMin) {
          done = true;
          break;
        }
        const float4 d = s3[buf][j];
        const float z = rho3 <= rho2 ? fmaf(c.w, u, fmaf(d.x, v, a.w)) : a.w;
        const float w = alpha * T;
        if (COUNT) ++ncontrib;
        C0 = fmaf(w, d.y, C0);
        C1 = fmaf(w, d.z, C1);
        C2 = fmaf(w, d.w, C2);
        D = fmaf(w, z, D);
        T = Tn;
      }
    }
  }
  cp_async_wait_all();

  if (inside) {
    const size_t p = (size_t)py * W + px, hw = (size_t)W * H;
    rgb[p] = fmaf(T, bg.x, C0);
    rgb[hw + p] = fmaf(T, bg.y, C1);
    rgb[2 * hw + p] = fmaf(T, bg.z, C2);
    if (depth) depth[p] = D;
    if (trans) trans[p] = T;
    if (MASKED && cls) cls[p] |= (uint8_t)kClsRender;
  }
  if (STATS) {
    // range of the alpha-normalised depth D / (1 - T) over pixels with coverage >= 0.5
    float lo = 3.0e38f, hi = 0.f;
    if (inside && 1.f - T >= 0.5f) {
      const float dh = D / (1.f - T);
      lo = dh;
      hi = dh;
    }
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
    unsigned long long v = npairs, c = ncontrib;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&ctr->pairs[eye], v);
      atomicAdd(&ctr->contrib[eye], c);
    }
  }
}

template <bool M, bool S, bool C>
static void launch_variant(int ntiles, cudaStream_t s, const Workspace &ws, const uint32_t *ids, int eye,
                           const uint8_t *mask, float3 bg, float *rgb, float *depth, float *trans, uint8_t *cls) {
  blend_kernel<M, S, C><<<ntiles, 256, 0, s>>>(ws.ranges, ids, ws.rec[eye], ws.cams, eye, mask, bg, rgb, depth,
                                               trans, cls, ws.ctr);
  GS_LAUNCHED(1);
}

cudaError_t launch_blend(const Workspace &ws, int eye, int W, int H, const uint8_t *tile_mask, float3 bg, float *rgb,
                         float *depth, float *trans, uint8_t *cls, bool depth_stats, bool count_pairs,
                         cudaStream_t s) {
  const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile, ntiles = tx * ty;
  if (ntiles == 0) return cudaSuccess;
  const uint32_t *ids = ws.ival[sorted_buffer(ntiles)];
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
