// Tile binning: an on-device LSD radix sort of packed (tile id | depth) keys.
//
// Paper: Sec. 3.1 Stage 1 and Sec. 3.5 (16x16 tiles of the 2DGS/3DGS tile
// rasterizer; Sec. 2.2 keeps its depth ordering).
//
// The sort key of an instance is (tile id << 32) | float_bits(z_c). Every
// instance of a surfel shares the depth digits, so the LSD passes over the low
// 32 bits run on the visible surfels *before* they are duplicated into
// instances, and only the tile digits are sorted per instance. LSD passes are
// stable, so this yields exactly the order of a full 64-bit LSD sort of the
// packed keys (ties broken by surfel index), with far less data moved.
//
// A surfel is binned to a tile only when its support can reach one of the
// tile's pixel centres: the support {o Ghat >= 1/255} is the union of the
// projected disc u^2 + v^2 <= r_c^2 (an ellipse in screen space, because the
// whole disc lies in front of the near plane) and the low-pass disc around the
// projected centre. The test is exact for the continuous tile rectangle (so it
// keeps every contributing pair) with the radius grown by 1e-3 for float32
// safety; the few surfels whose ellipse is too thin and oblique to solve in
// float32 keep their whole bounding rectangle.
//
// Pipeline per eye (all counts stay on the device):
//   1. count the tiles each surfel reaches (warp-cooperative; ROI-masked tiles
//      only when a mask is given)
//   2. compact the surfels with a non-zero count (scan) -> (depth bits, id)
//   3. radix sort over the 32 depth bits
//   4. scan of the counts in depth order -> instance offsets
//   5. emit (tile id, surfel id) in that order, coalesced per surfel
//   6. radix sort over the tile-id bits (stable: depth order kept per tile)
//   7. [start, end) range of every tile
#include "gs_internal.cuh"
#include "gs_scan.cuh"
#include "gs_sort.cuh"

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

// Tile columns [t0, t1] whose pixel centres meet the absolute interval [xa, xb].
__device__ __forceinline__ void tile_span(float xa, float xb, int W, int rx0, int rx1, int &t0, int &t1) {
  if (!(xa <= xb) || xa > (float)(W - 1) + kBoundPad || xb < -kBoundPad) {
    t0 = 1;
    t1 = 0;
    return;
  }
  t0 = max(rx0, (int)ceilf((xa - kBoundPad - (float)(kTile - 1)) * (1.f / kTile)));
  t1 = min(rx1, (int)floorf((xb + kBoundPad) * (1.f / kTile)));
}

// Up to two tile ranges [a0, a1] u [c0, c1] (disjoint, a before c) of tile row ty
// that the surfel's support reaches; empty ranges have lo > hi.
__device__ __forceinline__ void row_ranges(const Conic &q, const float4 r0, int ty, int W, int H, int rx0, int rx1,
                                           int &a0, int &a1, int &c0, int &c1) {
  const float y0 = (float)(ty * kTile) - kBoundPad;
  const float y1 = (float)min(ty * kTile + kTile - 1, H - 1) + kBoundPad;
  float elo, ehi, dlo, dhi;
  band_slices(q, y0 - r0.y, y1 - r0.y, elo, ehi, dlo, dhi);
  tile_span(r0.x + elo, r0.x + ehi, W, rx0, rx1, a0, a1);
  tile_span(r0.x + dlo, r0.x + dhi, W, rx0, rx1, c0, c1);
  if (a0 > a1) {
    a0 = c0; a1 = c1; c0 = 1; c1 = 0;
  } else if (c0 <= c1) {
    if (c0 <= a1 + 1 && c1 >= a0 - 1) {  // overlapping or adjacent: merge
      a0 = min(a0, c0); a1 = max(a1, c1); c0 = 1; c1 = 0;
    } else if (c1 < a0) {                 // keep the ranges in increasing order
      const int t0 = a0, t1 = a1;
      a0 = c0; a1 = c1; c0 = t0; c1 = t1;
    }
  }
}

// Tiles of [lo, hi] in tile row ty set in the ROI mask, from the row prefix
// counts mp[ty][x] = number of masked tiles of row ty left of column x.
__device__ __forceinline__ int masked_in(const uint16_t *mp, int tiles_x, int ty, int lo, int hi) {
  if (lo > hi) return 0;
  const uint16_t *row = mp + (size_t)ty * (tiles_x + 1);
  return (int)row[hi + 1] - (int)row[lo];
}

// Per-surfel tile count, one thread per surfel: rows of the bounding rectangle
// are walked with the closed-form ranges. A surfel whose screen ellipse is too
// thin and oblique for float32 (under 0.5% of surfels) keeps its whole bounding
// rectangle: binning more tiles than needed never changes the image, because
// the blend still evaluates alpha exactly, and it avoids a serial per-tile test.
__global__ void __launch_bounds__(256) count_kernel(uint32_t n, const float4 *__restrict__ rec,
                                                    const ushort4 *__restrict__ rect,
                                                    const uint32_t *__restrict__ aabb_cnt,
                                                    const uint8_t *__restrict__ mask, const uint16_t *__restrict__ mp,
                                                    const CamBlock *__restrict__ cams, int eye,
                                                    uint32_t *__restrict__ cnt_out) {
  const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  if (aabb_cnt[id] == 0u) {
    cnt_out[id] = 0u;
    return;
  }
  const int W = cams->eye[eye].W, H = cams->eye[eye].H, tiles_x = cams->eye[eye].tiles_x;
  const float4 *r = rec + 4 * (size_t)id;
  const float4 r0 = r[0], r1 = r[1], r2 = r[2];
  const ushort4 rc = rect[id];
  const Conic q = make_conic(r0, r1, r2);
  uint32_t count = 0;
  if (q.ok) {
    for (int ty = rc.y; ty <= rc.w; ++ty) {
      int a0, a1, c0, c1;
      row_ranges(q, r0, ty, W, H, rc.x, rc.z, a0, a1, c0, c1);
      if (mask) count += masked_in(mp, tiles_x, ty, a0, a1) + masked_in(mp, tiles_x, ty, c0, c1);
      else count += (uint32_t)(max(a1 - a0 + 1, 0) + max(c1 - c0 + 1, 0));
    }
  } else {
    for (int ty = rc.y; ty <= rc.w; ++ty)
      count += mask ? (uint32_t)masked_in(mp, tiles_x, ty, rc.x, rc.z) : (uint32_t)(rc.z - rc.x + 1);
  }
  cnt_out[id] = count;
}

// Emission, warp-cooperative: a warp takes one depth-sorted surfel at a time.
// Lane r computes the ranges of tile row r of a 32-row chunk; a warp scan of
// the row lengths gives every row's first slot, and each lane then fills slots
// lane, lane + 32, ..., finding its row by a binary search over the scan
// (consecutive lanes write consecutive slots). With a mask, rows are walked one
// by one and masked tiles compacted by ballot. Ill-conditioned ellipses take
// every tile of their rectangle (see count_kernel).
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t *__restrict__ ids, const uint32_t *n_ptr,
                                                   uint32_t n_max, const float4 *__restrict__ rec,
                                                   const ushort4 *__restrict__ rect, const uint8_t *__restrict__ mask,
                                                   const CamBlock *__restrict__ cams, int eye,
                                                   const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ offs,
                                                   uint32_t cap, uint32_t *__restrict__ ikey,
                                                   uint32_t *__restrict__ ival, uint32_t *__restrict__ n_sort) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n = load_n(n_ptr, n_max);
  const int W = cams->eye[eye].W, H = cams->eye[eye].H, tiles_x = cams->eye[eye].tiles_x;
  for (uint32_t j = warp; j < n; j += nwarps) {
    const uint32_t id = ids[j];
    const uint32_t base = offs[j];
    const uint32_t c = cnt[id];  // slots reserved for this surfel: never written past
    if ((uint64_t)base + c > cap) {
      // the first surfel that does not fit ends the binned instances
      if (lane == 0 && base <= cap) atomicMin(n_sort, base);
      continue;
    }
    const float4 *r = rec + 4 * (size_t)id;
    const float4 r0 = r[0], r1 = r[1], r2 = r[2];
    const ushort4 rc = rect[id];
    const int rows = rc.w - rc.y + 1;
    const Conic q = make_conic(r0, r1, r2);
    uint32_t count = 0;
    if (q.ok) {
      for (int rb = 0; rb < rows; rb += 32) {
        int a0 = 1, a1 = 0, c0 = 1, c1 = 0;
        if (rb + lane < rows) row_ranges(q, r0, rc.y + rb + lane, W, H, rc.x, rc.z, a0, a1, c0, c1);
        if (!mask) {
          const int len0 = max(a1 - a0 + 1, 0);
          const int len = len0 + max(c1 - c0 + 1, 0);
          int incl = len;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          // warp-uniform trip count: every lane takes part in the shuffles
          for (int s0 = 0; s0 < total; s0 += 32) {
            const int s = s0 + lane;
            // row of slot s: the first lane whose inclusive prefix exceeds s
            int lo = 0, hi = 31;
#pragma unroll
            for (int it = 0; it < 5; ++it) {
              const int mid = (lo + hi) >> 1;
              if (__shfl_sync(0xffffffffu, incl, mid) > s) hi = mid; else lo = mid + 1;
            }
            const int row = lo;
            const int before = __shfl_sync(0xffffffffu, incl - len, row);
            const int rs0 = __shfl_sync(0xffffffffu, a0, row);
            const int rl0 = __shfl_sync(0xffffffffu, len0, row);
            const int rt0 = __shfl_sync(0xffffffffu, c0, row);
            const int o = s - before;
            const int tx = o < rl0 ? rs0 + o : rt0 + (o - rl0);
            if (s < total && count + (uint32_t)s < c) {
              const uint32_t pos = base + count + (uint32_t)s;
              ikey[pos] = (uint32_t)((rc.y + rb + row) * tiles_x + tx);
              ival[pos] = id;
            }
          }
          count += (uint32_t)total;
          continue;
        }
        const int nr = min(32, rows - rb);
        for (int k = 0; k < nr; ++k) {
          const int ty_k = rc.y + rb + k;
          const int s0 = __shfl_sync(0xffffffffu, a0, k), s1 = __shfl_sync(0xffffffffu, a1, k);
          const int u0 = __shfl_sync(0xffffffffu, c0, k), u1 = __shfl_sync(0xffffffffu, c1, k);
          const int len0 = max(s1 - s0 + 1, 0), len = len0 + max(u1 - u0 + 1, 0);
          for (int t0 = 0; t0 < len; t0 += 32) {
            const int t = t0 + lane;
            bool hit = false;
            uint32_t tile = 0;
            if (t < len) {
              const int tx = t < len0 ? s0 + t : u0 + (t - len0);
              tile = (uint32_t)(ty_k * tiles_x + tx);
              hit = mask[tile] != 0;
            }
            const uint32_t ballot = __ballot_sync(0xffffffffu, hit);
            const uint32_t rank = count + __popc(ballot & lt);
            if (hit && rank < c) {
              ikey[base + rank] = tile;
              ival[base + rank] = id;
            }
            count += __popc(ballot);
          }
        }
      }
    } else {
      const int w = rc.z - rc.x + 1;
      const int total = w * rows;
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        bool hit = false;
        uint32_t tile = 0;
        if (t < total) {
          const int tx = rc.x + t % w, ty = rc.y + t / w;
          tile = (uint32_t)(ty * tiles_x + tx);
          hit = !mask || mask[tile];  // the whole rectangle, as counted
        }
        const uint32_t ballot = __ballot_sync(0xffffffffu, hit);
        const uint32_t rank = count + __popc(ballot & lt);
        if (hit && rank < c) {
          ikey[base + rank] = tile;
          ival[base + rank] = id;
        }
        count += __popc(ballot);
      }
    }
    // should a recount come out below the reserved slots, fill the rest with a
    // tile id past every real tile (sorted last, never ranged, never blended)
    for (uint32_t s = count + lane; s < c; s += 32) {
      ikey[base + s] = 0xffffffffu;
      ival[base + s] = id;
    }
  }
}

// Row prefix counts of the ROI tile mask: mp[ty][x] = masked tiles of row ty
// with column < x (one thread per row).
__global__ void mask_prefix_kernel(const uint8_t *__restrict__ mask, int tiles_x, int tiles_y, uint16_t *__restrict__ mp) {
  const int ty = blockIdx.x * blockDim.x + threadIdx.x;
  if (ty >= tiles_y) return;
  uint16_t *row = mp + (size_t)ty * (tiles_x + 1);
  int acc = 0;
  row[0] = 0;
  for (int tx = 0; tx < tiles_x; ++tx) {
    acc += mask[ty * tiles_x + tx] ? 1 : 0;
    row[tx + 1] = (uint16_t)acc;
  }
}

struct FlagLoad {
  const uint32_t *cnt;
  __device__ uint32_t operator()(uint32_t i) const { return cnt[i] > 0u ? 1u : 0u; }
};

struct CompactApply {
  const uint32_t *zkey;
  uint32_t *key_out, *val_out;
  uint32_t *n_out;
  __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t v) const {
    if (v) {
      key_out[prefix] = zkey[i];
      val_out[prefix] = i;
    }
  }
  __device__ void end(uint32_t, uint32_t total) const { *n_out = total; }
};

struct SortedCountLoad {
  const uint32_t *cnt;
  const uint32_t *ids;
  __device__ uint32_t operator()(uint32_t j) const { return cnt[ids[j]]; }
};

struct OffsetApply {
  uint32_t *offs;
  uint32_t *n_inst;
  uint32_t *n_sort;
  uint32_t cap;
  uint32_t *status;
  __device__ void operator()(uint32_t j, uint32_t prefix, uint32_t) const { offs[j] = prefix; }
  __device__ void end(uint32_t n, uint32_t total) const {
    offs[n] = total;
    *n_inst = total;
    *n_sort = total < cap ? total : cap;
    if (total > cap) atomicOr(status, kStCapacity);
  }
};

__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ n_ptr,
                                                     uint32_t ntiles, uint2 *__restrict__ ranges) {
  const uint32_t n = *n_ptr;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (t >= ntiles) continue;
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
  }
}

static int bits_for(int ntiles) {
  int b = 0;
  while ((1 << b) < ntiles) ++b;
  return b < 1 ? 1 : b;
}

// Buffer index holding the sorted instances: one pass per 8 tile bits, each pass
// flips between the two buffers.
int sorted_buffer(int ntiles) { return ((bits_for(ntiles) + 7) / 8) & 1; }

static int warp_grid(uint32_t n) {
  const uint32_t blocks = (n + 7) / 8;  // 8 warps per block, one surfel per warp
  return (int)(blocks < 1 ? 1 : (blocks > 152 * 16 ? 152 * 16 : blocks));
}

cudaError_t launch_binning(const Workspace &ws, int eye, int n, int tiles_x, int tiles_y,
                           const uint8_t *tile_mask, cudaStream_t s) {
  cudaError_t err;
  Counters *ctr = ws.ctr;
  const int ntiles = tiles_x * tiles_y;
  const uint32_t cap = (uint32_t)ws.max_instances;
  const RadixScratch rs{ws.rs_table, ws.rs_offs, ws.rs_n, ws.rs_sums};
  if ((err = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * (size_t)ntiles, s)) != cudaSuccess) return err;
  // 1. exact tile counts
  if (tile_mask) {
    mask_prefix_kernel<<<(tiles_y + 127) / 128, 128, 0, s>>>(tile_mask, tiles_x, tiles_y, ws.mask_prefix);
    GS_LAUNCHED(1);
  }
  if (n > 0) {
    count_kernel<<<(n + 255) / 256, 256, 0, s>>>((uint32_t)n, ws.rec[eye], ws.rect[eye], ws.cnt[eye], tile_mask,
                                                 ws.mask_prefix, ws.cams, eye, ws.cnt_bin);
    GS_LAUNCHED(1);
  }
  // 2. compact the binned surfels: (depth bits, surfel id)
  err = scan_launch(FlagLoad{ws.cnt_bin}, CompactApply{ws.zkey[eye], ws.dkey[0], ws.dval[0], &ctr->n_vis[eye]},
                    (const uint32_t *)nullptr, (uint32_t)n, ws.scan_sums, nullptr, s);
  if (err != cudaSuccess) return err;
  // 3. depth digits (the low 32 bits of the packed key)
  int which = 0;
  if ((err = radix_sort(ws.dkey, ws.dval, &ctr->n_vis[eye], (uint32_t)n, 32, rs, &which, s)) != cudaSuccess)
    return err;
  const uint32_t *ids = ws.dval[which];
  // 4. instance offsets in depth order
  err = scan_launch(SortedCountLoad{ws.cnt_bin, ids},
                    OffsetApply{ws.offs, &ctr->n_inst[eye], &ctr->n_sort[eye], cap, &ctr->status}, &ctr->n_vis[eye],
                    (uint32_t)n, ws.scan_sums, nullptr, s);
  if (err != cudaSuccess) return err;
  // 5. emission
  emit_kernel<<<warp_grid((uint32_t)n), 256, 0, s>>>(ids, &ctr->n_vis[eye], (uint32_t)n, ws.rec[eye], ws.rect[eye],
                                                     tile_mask, ws.cams, eye, ws.cnt_bin, ws.offs, cap, ws.ikey[0],
                                                     ws.ival[0], &ctr->n_sort[eye]);
  GS_LAUNCHED(1);
  // 6. tile digits (the high bits of the packed key)
  if ((err = radix_sort(ws.ikey, ws.ival, &ctr->n_sort[eye], cap, bits_for(ntiles), rs, &which, s)) != cudaSuccess)
    return err;
  // 7. ranges
  ranges_kernel<<<152 * 8, 256, 0, s>>>(ws.ikey[which], &ctr->n_sort[eye], (uint32_t)ntiles, ws.ranges);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace gs
