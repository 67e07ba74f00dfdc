// Persistent per-tile front-to-back alpha blending with the joint depth proxy.
//
// Paper: Sec. 3.1 Stage 1 - every contributing surfel gets the weight
// w_i = alpha_i T_i, and the same weight accumulates the colour C = sum c_i w_i
// and the depth proxy D = sum d_i w_i in one pass (no separate depth pass).
// Sec. 3.3 (Eq. 2 and the ray-splat intersection) gives alpha.
//
// One launch serves up to kRasterFrames (frame, eye) images - one eye of one
// frame, or one eye of every frame of a batch of scenes with different surfel
// counts and resolutions. The grid fills the SMs once; every CTA takes work
// items, (frame, tile) pairs numbered frame by frame, from a device counter
// until none is left, so the heavy tiles of one frame overlap the light tiles of
// the others and no CTA is launched per tile. A frame either offers every tile
// of its grid or a device list of tiles (the ROI tiles of a masked binning, or
// the masked 16-pixel tiles rendered from the lists of a coarser binning: each
// reads its parent tile's list, every surfel reaching the parent in depth
// order, and the surfels that miss its pixels contribute nothing).
//
// A CTA renders one TS x TS tile with TS^2 / PIX threads. A warp covers a block
// of 8 x (4 PIX) pixels (lane l: column l % 8, rows l / 8 + 4 q for q < PIX),
// so it can skip, in one uniform branch, every record whose screen bounds miss
// its block: those surfels cannot reach its pixels, and at 32-pixel tiles most
// of a tile's surfels reach only a few of its blocks. The homogeneous plane point p
// of a pixel is affine in the pixel offset (dx, dy) from the projected centre;
// the thread forms the dx terms once per surfel and adds the dy terms per pixel
// with three FMAs, so each surfel record read from shared memory serves PIX
// evaluations, and a pixel's arithmetic depends on its position only - not on
// the tile edge or block shape. The tile's depth-sorted surfel ids are
// consumed in batches of BATCH whose 64-byte records are staged in shared
// memory (structure of arrays: one broadcast float4 per field); cp.async
// double-buffers the next batch behind the current one. A tile ends as soon as
// all its pixels have terminated (__syncthreads_count). The result of a pixel
// does not depend on TS, PIX or BATCH: a tile's list holds every surfel whose
// support reaches any pixel centre of the tile, in depth order, and the others
// contribute nothing to its pixels.
//
// Ellipsoids (the 3DGS backbone) use the same loop: their record holds a
// Cholesky factor L of the screen conic Sigma2D^-1 = L^T L in place of the
// plane coefficients and a constant third coordinate, so the plane point is
// (L d, 1) and u^2 + v^2 = d^T Sigma2D^-1 d, the EWA exponent; the frame's
// low-pass factor is kNoLowpass (the EWA kernel already carries its 0.3 px^2
// filter) and the depth terms are zero, so every contribution has the centre
// depth.
#include "gs_internal.cuh"
#include "gs_launch.cuh"
#include "gs_scan.cuh"

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

// 1 / (2 ln 2): log2(o Ghat) = (r_c^2 - rho) / (2 ln 2) + log2(1/255)
constexpr float kHalfLog2e = 0.72134752044448170f;
// the row of a pixel that takes no more contributions
#define kNaN __int_as_float(0x7fffffff)

// The per-pixel part of one record's evaluation for a thread's PIX pixels of
// one column: dy = y - c_y, the plane point (qx, qy, qz) = (px0, py0, pz0) +
// dy (bz, bw, cz), u = qx / qz, v = qy / qz, rho3 = u^2 + v^2 and the low-pass
// term rho2 = lowpass (dx^2 + dy^2). Pixel pairs go through the packed FP32x2
// pipe (add/mul/fma .f32x2: one issue slot for two lanes' worth of work);
// every component is rounded exactly as the scalar operation, so the result
// does not depend on PIX.
template <int PIX>
__device__ __forceinline__ void eval_pixels(const float (&fy)[PIX], float ay, float bz, float bw, float cz,
                                            float px0, float py0, float pz0, float dx2, float lowpass,
                                            float (&uq)[PIX], float (&vq)[PIX], float (&r3q)[PIX],
                                            float (&r2q)[PIX]) {
  if constexpr (PIX % 2 == 0) {
    const float2 nay = make_float2(-ay, -ay), bz2 = make_float2(bz, bz), bw2 = make_float2(bw, bw);
    const float2 cz2 = make_float2(cz, cz), px2 = make_float2(px0, px0), py2 = make_float2(py0, py0);
    const float2 pz2 = make_float2(pz0, pz0), dx22 = make_float2(dx2, dx2), lp2 = make_float2(lowpass, lowpass);
#pragma unroll
    for (int p = 0; p < PIX / 2; ++p) {
      const float2 dy = __fadd2_rn(make_float2(fy[2 * p], fy[2 * p + 1]), nay);
      const float2 qx = __ffma2_rn(dy, bz2, px2);
      const float2 qy = __ffma2_rn(dy, bw2, py2);
      const float2 qz = __ffma2_rn(dy, cz2, pz2);
      const float2 iq = make_float2(rcp_approx(qz.x), rcp_approx(qz.y));
      const float2 u = __fmul2_rn(qx, iq), v = __fmul2_rn(qy, iq);
      const float2 r3 = __ffma2_rn(u, u, __fmul2_rn(v, v));
      const float2 r2 = __fmul2_rn(__ffma2_rn(dy, dy, dx22), lp2);
      uq[2 * p] = u.x; uq[2 * p + 1] = u.y;
      vq[2 * p] = v.x; vq[2 * p + 1] = v.y;
      r3q[2 * p] = r3.x; r3q[2 * p + 1] = r3.y;
      r2q[2 * p] = r2.x; r2q[2 * p + 1] = r2.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < PIX; ++q) {
      const float dy = fy[q] - ay;
      const float qx = fmaf(dy, bz, px0), qy = fmaf(dy, bw, py0), qz = fmaf(dy, cz, pz0);
      const float iq = rcp_approx(qz);
      uq[q] = qx * iq;
      vq[q] = qy * iq;
      r3q[q] = fmaf(uq[q], uq[q], vq[q] * vq[q]);
      r2q[q] = fmaf(dy, dy, dx2) * lowpass;
    }
  }
}

// Resident CTAs per SM asked of the compiler: with one or two pixels per thread
// the loop fits 64 registers, so 1024 threads (half the SM's warp slots) stay
// resident whatever the block shape (the 16-pixel shape otherwise takes 72 and
// keeps 7 CTAs of 128 threads); more pixels per thread keep their own count.
template <int TS, int PIX>
constexpr int raster_min_blocks() {
  return PIX <= 2 ? 1024 / (TS * TS / PIX) : 1;
}

template <int TS, int PIX, int BATCH, bool COUNT>
__global__ void __launch_bounds__(TS * TS / PIX, (raster_min_blocks<TS, PIX>()))
    raster_kernel(const __grid_constant__ RasterTable tab, uint32_t *__restrict__ queue) {
  griddep_wait();
  constexpr int NT = TS * TS / PIX;  // threads
  constexpr int RS = 4;              // rows between a thread's pixels
  constexpr int WBX = TS / 8;        // warp blocks per tile row
  static_assert(NT % 32 == 0 && PIX <= 8 && TS % 8 == 0 && TS % (4 * PIX) == 0, "block shape");
  __shared__ float4 s0[2][BATCH], s1[2][BATCH], s2[2][BATCH], s3[2][BATCH], s4[2][BATCH];
  __shared__ uint32_t s_first[kRasterFrames + 1];  // first work item of every frame
  __shared__ uint32_t s_item[2];                   // double-buffered: one barrier per item

  if (threadIdx.x < 32) {
    const int f = threadIdx.x;
    uint32_t c = 0;
    if (f < tab.n) {
      const RasterFrame &fr = tab.f[f];
      c = (uint32_t)fr.ntiles;
      if (fr.items) c = min(c, *fr.n_items);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, c, o);
      if (f >= o) c += y;
    }
    s_first[f + 1] = c;
    if (f == 0) s_first[0] = 0u;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx0 = (warp % WBX) * 8, by0 = (warp / WBX) * (4 * PIX);  // the warp's block in the tile
  const int lx = bx0 + (lane & 7), ly = by0 + (lane >> 3);

  if (threadIdx.x == 0) s_item[0] = atomicAdd(queue, 1u);
  for (int it = 0;; it ^= 1) {
    // orders the item (and, the first time, s_first) before its reads, and every
    // read of the previous tile's shared records before this tile's staging
    __syncthreads();
    const uint32_t g = s_item[it];
    if (g >= s_first[tab.n]) break;  // CTA-uniform
    int f = 0;
    while (f + 1 < tab.n && s_first[f + 1] <= g) ++f;
    const RasterFrame &fr = tab.f[f];
    const uint32_t k = g - s_first[f];
    const int tile = fr.items ? (int)fr.items[k] : (int)k;

    const int W = fr.W, H = fr.H;
    const int px = (tile % fr.tiles_x) * TS + lx;
    const int py = (tile / fr.tiles_x) * TS + ly;  // first of rows py, py + RS, ...
    // a tile of a finer grid than the binning's reads its parent tile's list
    // (every surfel reaching the parent, a superset of the tile's own)
    const int rt = fr.rshift ? ((tile / fr.tiles_x) >> fr.rshift) * fr.rtiles_x + ((tile % fr.tiles_x) >> fr.rshift)
                             : tile;
    const uint2 rg = fr.ranges[rt];
    const int rtx = (W + kTile - 1) / kTile;

    const float fx = (float)px;
    const float lowpass = fr.lowpass;
    // the warp's pixel block (pixel centres), for the record culling
    const float wx0 = (float)((tile % fr.tiles_x) * TS + bx0), wy0 = (float)((tile / fr.tiles_x) * TS + by0);
    const float wx1 = wx0 + 7.f, wy1 = wy0 + (float)(4 * PIX - 1);
    // the thread's pixel rows; a pixel that is not blending (outside the image
    // or the ROI, or finished) has a NaN row, so every test on it fails
    float fy[PIX];
    float T[PIX], C0[PIX], C1[PIX], C2[PIX], D[PIX];
    unsigned live = 0;  // bit k: pixel k still blending
#pragma unroll
    for (int q = 0; q < PIX; ++q) {
      T[q] = 1.f; C0[q] = C1[q] = C2[q] = D[q] = 0.f;
      const int y = py + RS * q;
      bool on = px < W && y < H;
      if (on && fr.roi) on = fr.roi[(y / kTile) * rtx + px / kTile] != 0;
      if (on && fr.skip) on = fr.skip[(y / kTile) * rtx + px / kTile] == 0;
      fy[q] = on ? (float)y : kNaN;
      if (on) live |= 1u << q;
    }
    const unsigned wmask = live;  // pixels this thread writes
    unsigned npairs = 0, ncontrib = 0;

    auto stage = [&](int buf, uint32_t b0) {
      for (int slot = threadIdx.x; slot < BATCH; slot += NT) {
        const uint32_t i = b0 + (uint32_t)slot;
        if (i < rg.y) {
          const uint32_t id = fr.ids[i];
          if (id < fr.n_rec) {
            const float4 *r = fr.rec + 4 * (size_t)id;
            cp_async16(&s0[buf][slot], r + 0);
            cp_async16(&s1[buf][slot], r + 1);
            cp_async16(&s2[buf][slot], r + 2);
            cp_async16(&s3[buf][slot], r + 3);
            cp_async16(&s4[buf][slot], fr.box + id);
          } else {  // never expected; a record that cannot contribute keeps reads in bounds
            s0[buf][slot] = make_float4(0.f, 0.f, -1.f, 1.f);
            s1[buf][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
            s2[buf][slot] = make_float4(1.f, 0.f, 0.f, 0.f);
            s3[buf][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
            s4[buf][slot] = make_float4(1.f, 0.f, 1.f, 0.f);  // empty bounds
          }
        }
      }
      cp_async_commit();
    };

    int buf = 0;
    if (rg.x < rg.y) stage(0, rg.x);
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += BATCH, buf ^= 1) {
      cp_async_wait_all();
      // barrier: the batch in `buf` is visible to all, and every thread has
      // finished reading the other buffer, which the prefetch below overwrites
      if (__syncthreads_count(live == 0u) == NT) break;
      if (b0 + BATCH < rg.y) stage(buf ^ 1, b0 + BATCH);
      const int nb = (int)min((uint32_t)BATCH, rg.y - b0);
#pragma unroll 4
      for (int j = 0; j < nb && live; ++j) {
        // warp-uniform: the record's bounds miss the warp's block
        const float4 bb = s4[buf][j];
        if (bb.y < wx0 || bb.x > wx1 || bb.w < wy0 || bb.z > wy1) continue;
        const float4 a = s0[buf][j];
        const float4 b = s1[buf][j];
        const float4 c = s2[buf][j];
        // homogeneous plane point p = (dx b.x + dy b.z, dx b.y + dy b.w,
        // c.x + dx c.y + dy c.z): the column's dx terms, then dy per pixel
        const float dx = fx - a.x;
        const float px0 = dx * b.x, py0 = dx * b.y, pz0 = fmaf(dx, c.y, c.x);
        const float dx2 = dx * dx;
        // per pixel: u, v, rho3 and the low-pass term rho2 = lowpass |x - c|^2
        float uq[PIX], vq[PIX], r3q[PIX], r2q[PIX];
        eval_pixels<PIX>(fy, a.y, b.z, b.w, c.z, px0, py0, pz0, dx2, lowpass, uq, vq, r3q, r2q);
#pragma unroll
        for (int q = 0; q < PIX; ++q) {
          const float rho3 = r3q[q], rho2 = r2q[q];
          const float rho = fminf(rho3, rho2);
          if (COUNT && (live & (1u << q))) ++npairs;
          if (rho <= a.z) {  // alpha >= 1/255 (false for a NaN row)
            const float alpha = fminf(kAlphaMax, ex2_approx(fmaf(a.z - rho, kHalfLog2e, kLog2AlphaMin)));
            const float Tn = fmaf(-T[q], alpha, T[q]);
            if (Tn < kTMin) {
              live &= ~(1u << q);
              fy[q] = kNaN;
            } else {
              const float4 d = s3[buf][j];
              const float z = rho3 <= rho2 ? fmaf(c.w, uq[q], fmaf(d.x, vq[q], a.w)) : a.w;
              const float w = alpha * T[q];
              if (COUNT) ++ncontrib;
              C0[q] = fmaf(w, d.y, C0[q]);
              C1[q] = fmaf(w, d.z, C1[q]);
              C2[q] = fmaf(w, d.w, C2[q]);
              D[q] = fmaf(w, z, D[q]);
              T[q] = Tn;
            }
          }
        }
      }
    }
    cp_async_wait_all();
    // the next item: its round trip overlaps the output stores below
    uint32_t next = 0;
    if (threadIdx.x == 0) next = atomicAdd(queue, 1u);

    const size_t hw = (size_t)W * H;
    float lo = 3.0e38f, hi = 0.f;
#pragma unroll
    for (int q = 0; q < PIX; ++q) {
      if (!(wmask & (1u << q))) continue;
      const size_t p = (size_t)(py + RS * q) * W + px;
      fr.rgb[p] = fmaf(T[q], fr.bg[0], C0[q]);
      fr.rgb[hw + p] = fmaf(T[q], fr.bg[1], C1[q]);
      fr.rgb[2 * hw + p] = fmaf(T[q], fr.bg[2], C2[q]);
      if (fr.depth) fr.depth[p] = D[q];
      if (fr.trans) fr.trans[p] = T[q];
      if (fr.winit) fr.winit[p] = kNoSample;
      if (fr.cls) fr.cls[p] |= (uint8_t)kClsRender;
      if (1.f - T[q] >= 0.5f) {
        // range of the alpha-normalised depth D / (1 - T) over pixels with coverage >= 0.5
        const float dh = D[q] / (1.f - T[q]);
        lo = fminf(lo, dh);
        hi = fmaxf(hi, dh);
      }
    }
    if (fr.stats) {  // CTA-uniform
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if ((threadIdx.x & 31) == 0 && hi > 0.f) {
        atomicMin(&fr.ctr->dmin_bits, __float_as_uint(fmaxf(lo, 0.f)));
        atomicMax(&fr.ctr->dmax_bits, __float_as_uint(hi));
      }
    }
    if (threadIdx.x == 0) s_item[it ^ 1] = next;  // read after the next barrier
    if (COUNT) {
      unsigned long long v = npairs, cc = ncontrib;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        cc += __shfl_xor_sync(0xffffffffu, cc, o);
      }
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(&fr.ctr->pairs[fr.eye], v);
        atomicAdd(&fr.ctr->contrib[fr.eye], cc);
      }
    }
  }
  // the last CTA out clears the counter and the ticket for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
      queue[0] = 0u;
      queue[1] = 0u;
    }
  }
}

// ---------------------------------------------------------------- work order
// Longest tile lists first. The persistent rasterizer takes its work items in
// list order, so a frame whose heaviest tiles come last ends on a few CTAs
// still walking long lists while the other SMs idle. One CTA counting-sorts the
// frame's items by a log-scale bucket of their surfel-list length (eight
// buckets per octave, longest first; the order inside a bucket is arbitrary).
// The order changes no pixel: every item renders its own pixels.
constexpr int kLptThreads = 1024;

__device__ __forceinline__ uint32_t lpt_bucket(uint32_t len) {
  const uint32_t v = len + 1u;
  const uint32_t lg = 31u - (uint32_t)__clz(v);
  const uint32_t frac = lg >= 3u ? (v >> (lg - 3u)) & 7u : (v << (3u - lg)) & 7u;
  return 255u - min(255u, lg * 8u + frac);
}

__global__ void __launch_bounds__(kLptThreads) lpt_order_kernel(const uint32_t *__restrict__ items,
                                                                const uint32_t *n_items, uint32_t n_max,
                                                                const uint2 *__restrict__ ranges, int tiles_x,
                                                                int rshift, int rtiles_x, uint32_t *__restrict__ out) {
  griddep_wait();
  __shared__ uint32_t s_hist[256];
  __shared__ uint32_t s_scan[32];
  const uint32_t n = items ? min(*n_items, n_max) : n_max;
  auto bucket = [&](uint32_t k, uint32_t &tile) {
    tile = items ? items[k] : k;
    const uint32_t rt = rshift ? (tile / (uint32_t)tiles_x >> rshift) * (uint32_t)rtiles_x +
                                     (tile % (uint32_t)tiles_x >> rshift)
                               : tile;
    const uint2 rg = ranges[rt];
    return lpt_bucket(rg.y - rg.x);
  };
  if (threadIdx.x < 256) s_hist[threadIdx.x] = 0u;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < n; k += kLptThreads) {
    uint32_t t;
    atomicAdd(&s_hist[bucket(k, t)], 1u);
  }
  __syncthreads();
  uint32_t base;
  block_exclusive_scan<kLptThreads>(threadIdx.x < 256 ? s_hist[threadIdx.x] : 0u, &base, s_scan);
  __syncthreads();
  if (threadIdx.x < 256) s_hist[threadIdx.x] = base;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < n; k += kLptThreads) {
    uint32_t t;
    const uint32_t b = bucket(k, t);
    out[1u + atomicAdd(&s_hist[b], 1u)] = t;
  }
  if (threadIdx.x == 0) out[0] = n;
}

// ---------------------------------------------------------------- host side

namespace {

struct Variant {
  const void *fn;
  int threads;
  int occupancy;  // resident CTAs per SM, 0 until queried
};

constexpr int kShapes = 7;  // (tile, pix): (8,1) (8,2) (16,2) (16,4) (32,4) (32,8) (32,2)
constexpr int kBatches = 4; // 32 64 128 256

template <int TS, int PIX, bool C>
void fill_batches(Variant *v) {
  v[0] = Variant{(const void *)raster_kernel<TS, PIX, 32, C>, TS * TS / PIX, 0};
  v[1] = Variant{(const void *)raster_kernel<TS, PIX, 64, C>, TS * TS / PIX, 0};
  v[2] = Variant{(const void *)raster_kernel<TS, PIX, 128, C>, TS * TS / PIX, 0};
  v[3] = Variant{(const void *)raster_kernel<TS, PIX, 256, C>, TS * TS / PIX, 0};
}

struct VariantTable {
  Variant v[2][kShapes][kBatches];
  VariantTable() {
    fill_batches<8, 1, false>(v[0][0]);
    fill_batches<8, 2, false>(v[0][1]);
    fill_batches<16, 2, false>(v[0][2]);
    fill_batches<16, 4, false>(v[0][3]);
    fill_batches<32, 4, false>(v[0][4]);
    fill_batches<32, 8, false>(v[0][5]);
    fill_batches<32, 2, false>(v[0][6]);
    fill_batches<8, 1, true>(v[1][0]);
    fill_batches<8, 2, true>(v[1][1]);
    fill_batches<16, 2, true>(v[1][2]);
    fill_batches<16, 4, true>(v[1][3]);
    fill_batches<32, 4, true>(v[1][4]);
    fill_batches<32, 8, true>(v[1][5]);
    fill_batches<32, 2, true>(v[1][6]);
  }
};

VariantTable g_variants;

int shape_index(const RasterConfig &c) {
  switch (c.tile) {
    case 8: return c.pix == 1 ? 0 : c.pix == 2 ? 1 : -1;
    case 16: return c.pix == 2 ? 2 : c.pix == 4 ? 3 : -1;
    case 32: return c.pix == 4 ? 4 : c.pix == 8 ? 5 : c.pix == 2 ? 6 : -1;
  }
  return -1;
}

int batch_index(int b) { return b == 32 ? 0 : b == 64 ? 1 : b == 128 ? 2 : b == 256 ? 3 : -1; }

}  // namespace

int sm_count() {
  static int cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
  if (dev < 64 && cached[dev] > 0) return cached[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev < 64) cached[dev] = n;
  return n;
}

bool raster_config_ok(const RasterConfig &c) { return shape_index(c) >= 0 && batch_index(c.batch) >= 0; }

int raster_tshift(const RasterConfig &c) { return c.tile == 8 ? 3 : c.tile == 32 ? 5 : 4; }

cudaError_t launch_raster(const RasterTable &t, const RasterConfig &c, bool count_pairs, uint32_t *queue,
                          cudaStream_t s) {
  if (!raster_config_ok(c) || t.n < 0 || t.n > kRasterFrames) return cudaErrorInvalidValue;
  if (t.n == 0) return cudaSuccess;
  Variant &v = g_variants.v[count_pairs ? 1 : 0][shape_index(c)][batch_index(c.batch)];
  if (v.occupancy <= 0) {
    int occ = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, v.threads, 0);
    if (e != cudaSuccess) return e;
    v.occupancy = occ > 0 ? occ : 1;
  }
  const int sms = sm_count();
  if (sms <= 0) return cudaErrorNoDevice;
  RasterTable arg = t;
  void *args[2] = {(void *)&arg, (void *)&queue};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3((unsigned)(sms * v.occupancy));
  cfg.blockDim = dim3((unsigned)v.threads);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelExC(&cfg, v.fn, args);
  GS_LAUNCHED(1);
  return e;
}

cudaError_t launch_lpt_order(RasterFrame &f, uint32_t *buf, cudaStream_t s) {
  const cudaError_t e = launch_k(lpt_order_kernel, 1, kLptThreads, 0, s, f.items, f.n_items, (uint32_t)f.ntiles,
                                 f.ranges, f.tiles_x, f.rshift, f.rtiles_x, buf);
  GS_LAUNCHED(1);
  f.items = buf + 1;
  f.n_items = buf;
  return e;
}

RasterFrame raster_frame(const Workspace &ws, int eye, int W, int H, int tshift, const uint8_t *mask, float3 bg,
                         float *rgb, float *depth, float *trans, uint8_t *cls, bool stats) {
  RasterFrame f;
  const int ts = 1 << tshift;
  f.ranges = ws.bin[eye].ranges;
  f.ids = ws.bin[eye].ival;
  f.rec = ws.rec[eye];
  f.box = ws.bounds[eye];
  f.roi = (mask && tshift > 4) ? mask : nullptr;  // a 32-pixel tile may hold unmasked 16-pixel tiles
  f.skip = nullptr;
  f.rshift = 0;
  f.rtiles_x = 0;
  f.items = mask ? ws.bin[eye].items : nullptr;
  f.n_items = mask ? &ws.ctr->n_items[eye] : nullptr;
  f.rgb = rgb;
  f.depth = depth;
  f.trans = trans;
  f.cls = cls;
  f.winit = nullptr;
  f.ctr = ws.ctr;
  f.bg[0] = bg.x;
  f.bg[1] = bg.y;
  f.bg[2] = bg.z;
  f.W = W;
  f.H = H;
  f.tiles_x = (W + ts - 1) >> tshift;
  f.ntiles = f.tiles_x * ((H + ts - 1) >> tshift);
  f.tshift = tshift;
  f.eye = eye;
  f.stats = stats ? 1 : 0;
  f.lowpass = ws.prim ? kNoLowpass : 2.f;
  f.n_rec = (uint32_t)ws.max_surfels;
  return f;
}


}  // namespace gs
