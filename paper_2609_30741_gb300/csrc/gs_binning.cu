// Tile binning: every tile's list of the surfels that can reach it, in the
// order of the packed (tile id | depth) key sort of the 2DGS/3DGS tile
// rasterizer.
//
// Paper: Sec. 3.1 Stage 1 and Sec. 3.5 (16x16 tiles of the 2DGS/3DGS tile
// rasterizer; Sec. 2.2 keeps its depth ordering).
//
// Sorting by (tile, depth) is the same as sorting the surfels by depth first and
// then grouping them by tile without changing their order. So the surfels are
// radix sorted once on their 32 depth bits (ties keep the index order), and
// the grouping by tile is a stable counting sort: the depth-ordered surfels are
// cut into chunks, a first pass counts each chunk's hits per tile into a
// [tile][chunk] table, one scan of that table gives every (tile, chunk) run its
// place, and a second pass writes the surfel ids straight into their slots. The
// per-instance (tile, surfel) pairs are never materialised or radix sorted.
//
// A surfel is binned to a tile only when its support can reach one of the
// tile's pixel centres: the support {o Ghat >= 1/255} is the union of the
// projected disc u^2 + v^2 <= r_c^2 (an ellipse in screen space, because the
// whole disc lies in front of the near plane) and the low-pass disc around the
// projected centre. The test is exact for the continuous tile rectangle (so it
// keeps every contributing pair) with the radius grown by 1e-3 for float32
// safety; the few surfels whose ellipse is too thin and oblique to solve in
// float32 keep their whole bounding rectangle. An ellipsoid's record has the
// same form (its screen conic in place of the plane coefficients) and no
// low-pass disc.
//
// Pipeline per eye (all counts stay on the device):
//   1. compact the surfels with a non-empty rectangle (reaching an ROI tile when
//      a mask is given) -> (depth bits, id)
//   2. tile ranges of every rectangle row of those surfels (rows_kernel)
//   3. radix sort over the 32 depth bits
//   4. per-chunk, per-warp lists of the surfels reaching each band of tile rows
//   5. per-(tile, chunk) counts (bin_kernel, mode 0)
//   6. tile-major scan of the counts -> run offsets, tile ranges
//   7. placement of every surfel id (bin_kernel, mode 1)
#include <mutex>

#include "gs_conic.cuh"
#include "gs_internal.cuh"
#include "gs_launch.cuh"
#include "gs_scan.cuh"
#include "gs_sort.cuh"

namespace gs {

// Tile columns [t0, t1] (tile edge ts = 1 << tshift) whose pixel centres meet the
// absolute interval [xa, xb].
__device__ __forceinline__ void tile_span(float xa, float xb, int W, int rx0, int rx1, int tshift, int &t0,
                                          int &t1) {
  if (!(xa <= xb) || xa > (float)(W - 1) + kBoundPad || xb < -kBoundPad) {
    t0 = 1;
    t1 = 0;
    return;
  }
  const float ts = (float)(1 << tshift), its = 1.f / ts;  // exact: a power of two
  t0 = max(rx0, (int)ceilf((xa - kBoundPad - (ts - 1.f)) * its));
  t1 = min(rx1, (int)floorf((xb + kBoundPad) * its));
}

// Up to two tile ranges [a0, a1] u [c0, c1] (disjoint, a before c) of tile row ty
// that the surfel's support reaches; empty ranges have lo > hi.
__device__ __forceinline__ void row_ranges(const Conic &q, const float4 r0, int ty, int W, int H, int rx0, int rx1,
                                           int tshift, int &a0, int &a1, int &c0, int &c1) {
  const int ts = 1 << tshift;
  const float y0 = (float)(ty * ts) - kBoundPad;
  const float y1 = (float)min(ty * ts + ts - 1, H - 1) + kBoundPad;
  float elo, ehi, dlo, dhi;
  band_slices(q, y0 - r0.y, y1 - r0.y, elo, ehi, dlo, dhi);
  tile_span(r0.x + elo, r0.x + ehi, W, rx0, rx1, tshift, a0, a1);
  tile_span(r0.x + dlo, r0.x + dhi, W, rx0, rx1, tshift, c0, c1);
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

// Summed-area table of the ROI tile mask: sat[y][x] = masked tiles with row < y
// and column < x, (tiles_y + 1) x (tiles_x + 1) entries. One block: each warp
// takes whole rows (prefix counts by ballot, 32 columns at a time), then each
// thread adds one column down the rows.
// With roi16 given, the mask is first derived from the ROI mask on the 16-pixel
// grid (rtx x rty tiles): a tile of edge 1 << tshift is masked when it holds a
// masked pixel. clip[0][ty][tx] / clip[1][ty][tx] get the first masked column
// >= tx / the last masked column <= tx of row ty (0xffff: none), by ballots 32
// columns at a time with the carry of the columns already passed. With list16
// given, list16[0] gets the number of masked 16-pixel tiles and list16[1..] the
// tiles (a rasterizer on the 16-pixel grid reading this grid's lists).
__global__ void __launch_bounds__(1024) mask_sat_kernel(uint8_t *mask, int tiles_x, int tiles_y,
                                                        uint32_t *__restrict__ sat, const uint8_t *__restrict__ roi16,
                                                        int rtx, int rty, int tshift, uint16_t *__restrict__ clip,
                                                        uint32_t *__restrict__ list16) {
  griddep_wait();
  constexpr int kSatSmem = 12000;
  __shared__ uint32_t s_sat[kSatSmem];
  __shared__ uint32_t s_n16;
  if (list16 && roi16) {
    if (threadIdx.x == 0) s_n16 = 0u;
    __syncthreads();
    const int n16 = rtx * rty;
    for (int b0 = (threadIdx.x >> 5) * 32; b0 < n16; b0 += (int)blockDim.x) {  // warp-uniform
      const int t = b0 + (int)(threadIdx.x & 31);
      const bool on = t < n16 && roi16[t] != 0;
      const unsigned bal = __ballot_sync(0xffffffffu, on);
      if (!bal) continue;
      uint32_t base = 0;
      if ((threadIdx.x & 31) == 0) base = atomicAdd(&s_n16, (uint32_t)__popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (on) list16[1 + base + (uint32_t)__popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = (uint32_t)t;
    }
    __syncthreads();
    if (threadIdx.x == 0) list16[0] = s_n16;
  }
  if (roi16) {
    for (int t = threadIdx.x; t < tiles_x * tiles_y; t += blockDim.x) {
      const int x = t % tiles_x, y = t / tiles_x;
      uint8_t v = 0;
      if (tshift <= 4) {
        v = roi16[(y >> (4 - tshift)) * rtx + (x >> (4 - tshift))];
      } else {
        const int sc = 1 << (tshift - 4);
        for (int dy = 0; dy < sc; ++dy)
          for (int dx = 0; dx < sc; ++dx) {
            const int yy = y * sc + dy, xx = x * sc + dx;
            if (yy < rty && xx < rtx) v |= roi16[yy * rtx + xx];
          }
      }
      mask[t] = v ? 1 : 0;
    }
    __syncthreads();
  }
  const int sx = tiles_x + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nt = tiles_x * tiles_y;
  for (int y = wid; y < tiles_y; y += nw) {
    const uint8_t *row = mask + (size_t)y * tiles_x;
    uint32_t carry = 0xffffu;  // previous masked column: left to right
    for (int x0 = 0; x0 < tiles_x; x0 += 32) {  // warp-uniform
      const int x = x0 + lane;
      const uint32_t b = __ballot_sync(0xffffffffu, x < tiles_x && row[x] != 0);
      const uint32_t le = b & (0xffffffffu >> (31 - lane));  // columns <= x
      if (x < tiles_x) clip[nt + y * tiles_x + x] = (uint16_t)(le ? (uint32_t)x0 + 31u - __clz(le) : carry);
      if (b) carry = (uint32_t)x0 + 31u - __clz(b);
    }
    carry = 0xffffu;  // next masked column: right to left
    for (int x0 = (tiles_x - 1) & ~31; x0 >= 0; x0 -= 32) {  // warp-uniform
      const int x = x0 + lane;
      const uint32_t b = __ballot_sync(0xffffffffu, x < tiles_x && row[x] != 0);
      const uint32_t ge = b & (0xffffffffu << lane);  // columns >= x
      if (x < tiles_x) clip[y * tiles_x + x] = (uint16_t)(ge ? (uint32_t)x0 + (uint32_t)__ffs(ge) - 1u : carry);
      if (b) carry = (uint32_t)x0 + (uint32_t)__ffs(b) - 1u;
    }
  }
  // the table is built in shared memory when it fits (the column pass is a
  // dependent chain down each column) and then copied out
  const int nsat = (tiles_y + 1) * sx;
  uint32_t *S = nsat <= kSatSmem ? s_sat : sat;
  for (int y = wid; y <= tiles_y; y += nw) {
    uint32_t acc = 0;
    if (lane == 0) S[(size_t)y * sx] = 0u;
    for (int x0 = 0; x0 < tiles_x; x0 += 32) {  // warp-uniform
      const int x = x0 + lane;
      const bool on = y > 0 && x < tiles_x && mask[(size_t)(y - 1) * tiles_x + x] != 0;
      const uint32_t b = __ballot_sync(0xffffffffu, on);
      if (x < tiles_x) S[(size_t)y * sx + x + 1] = acc + (uint32_t)__popc(b & (0xffffffffu >> (31 - lane)));
      acc += (uint32_t)__popc(b);
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x <= tiles_x; x += blockDim.x) {
    uint32_t acc = 0;
    for (int y = 1; y <= tiles_y; ++y) {
      acc += S[(size_t)y * sx + x];
      S[(size_t)y * sx + x] = acc;
    }
  }
  if (S != sat) {
    __syncthreads();
    for (int i = threadIdx.x; i < nsat; i += blockDim.x) sat[i] = S[i];
  }
}

// Any ROI tile in tile rows [y0, y1] x columns [x0, x1]?
__device__ __forceinline__ bool sat_any(const uint32_t *sat, int tiles_x, int y0, int y1, int x0, int x1) {
  if (y0 > y1 || x0 > x1) return false;
  const int sx = tiles_x + 1;
  const uint32_t v = sat[(size_t)(y1 + 1) * sx + x1 + 1] - sat[(size_t)y0 * sx + x1 + 1] -
                     sat[(size_t)(y1 + 1) * sx + x0] + sat[(size_t)y0 * sx + x0];
  return v != 0u;
}

// The masked tiles of tile row ty between columns [x0, x1]: the span clipped to
// its first and last masked tile (empty, lo > hi, when it has none), from the
// row's next / previous masked-column tables. The tiles in between may still be
// unmasked; the counting sort skips those one by one.
__device__ __forceinline__ void clip_to_mask(const uint16_t *clip, int tiles_x, int tiles_y, int ty, int &x0,
                                             int &x1) {
  if (x0 > x1) return;
  const int first = clip[ty * tiles_x + x0];  // 0xffff when none: beyond any column
  if (first > x1) {
    x0 = 1;
    x1 = 0;
    return;
  }
  x1 = clip[tiles_x * tiles_y + ty * tiles_x + x1];
  x0 = first;
}

// ---------------------------------------------------------------- row spans
// Once per eye and frame, every tile row of every surfel's bounding rectangle
// gets its tile ranges [a0, a1] u [c0, c1] (row_ranges; an ill-conditioned
// ellipse keeps the whole row of its rectangle), packed as 4 x 16 bits. A warp
// takes 32 consecutive surfels (one per lane), reserves slots for all their rows
// with one atomic, and then computes the rows 32 at a time, one per lane, so no
// lane idles while another walks a large surfel. row_off[i] is the slot of
// surfel i's first rectangle row. An ROI binning keeps of each range only the
// part from its first to its last masked tile. The grid strides over the
// surfels, so a small grid can run beside other kernels; without ids the
// candidates are all surfels by id, and with the ROI's summed-area table a
// surfel whose rectangle holds no ROI tile is skipped (the compaction's test),
// so the spans need neither the compaction nor the depth order.
__global__ void __launch_bounds__(256) rows_kernel(const uint32_t *__restrict__ ids, const uint32_t *n_ptr,
                                                   uint32_t n_max, const float4 *__restrict__ rec,
                                                   const ushort4 *__restrict__ rect, const uint32_t *__restrict__ cnt,
                                                   const CamBlock *__restrict__ cams, int eye, int prim,
                                                   uint32_t *__restrict__ row_off, uint2 *__restrict__ spans,
                                                   uint32_t cap, uint32_t *__restrict__ n_rows,
                                                   uint32_t *__restrict__ status, const uint16_t *__restrict__ clip,
                                                   int clip_tiles_x, int clip_tiles_y,
                                                   const uint32_t *__restrict__ sat) {
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const uint32_t n = load_n(n_ptr, n_max);
  const int W = cams->eye[eye].W, H = cams->eye[eye].H, tshift = cams->eye[eye].tshift;
  const uint32_t stride = gridDim.x * blockDim.x;  // a multiple of 32: j0 stays warp-aligned
  for (uint32_t j0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; j0 < n; j0 += stride) {  // warp-uniform
  const uint32_t j = j0 + (uint32_t)lane;
  const uint32_t i = j < n ? (ids ? ids[j] : j) : 0u;  // the surfels being binned
  int nr = 0, ry = 0, rx0 = 0, rx1 = -1;
  Conic q{};
  float cx = 0.f, cy = 0.f;
  bool bin = j < n && cnt[i] > 0u;
  ushort4 rc = make_ushort4(0, 0, 0, 0);
  if (bin) {
    rc = rect[i];
    if (sat) bin = sat_any(sat, clip_tiles_x, rc.y, rc.w, rc.x, rc.z);  // the binning's ROI test
  }
  if (bin) {
    nr = (int)rc.w - (int)rc.y + 1;
    ry = rc.y;
    rx0 = rc.x;
    rx1 = rc.z;
    const float4 *r = rec + 4 * (size_t)i;
    const float4 r0 = r[0], r1 = r[1], r2 = r[2];
    q = make_conic(r0, r1, r2);
    if (prim) q.rl2 = -1.f;  // ellipsoids have no low-pass disc
    cx = r0.x;
    cy = r0.y;
  }
  int incl = nr;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  uint32_t base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(n_rows, (uint32_t)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  if (lane == 0 && total > 0 && (uint64_t)base + (uint64_t)total > cap) atomicOr(status, kStCapacity);
  if (j < n) row_off[i] = base + (uint32_t)(incl - nr);
  for (int q0 = 0; q0 < total; q0 += 32) {
    const int qq = q0 + lane;
    int kl = 0, kh = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const int mid = (kl + kh) >> 1;
      if (__shfl_sync(0xffffffffu, incl, mid) > qq) kh = mid; else kl = mid + 1;
    }
    const int k = kl;
    const int excl_k = __shfl_sync(0xffffffffu, incl, k) - __shfl_sync(0xffffffffu, nr, k);
    const int ty = __shfl_sync(0xffffffffu, ry, k) + (qq - excl_k);
    const int sx0 = __shfl_sync(0xffffffffu, rx0, k), sx1 = __shfl_sync(0xffffffffu, rx1, k);
    Conic qk;
    qk.Sxx = __shfl_sync(0xffffffffu, q.Sxx, k);
    qk.Sxy = __shfl_sync(0xffffffffu, q.Sxy, k);
    qk.Syy = __shfl_sync(0xffffffffu, q.Syy, k);
    qk.gx = __shfl_sync(0xffffffffu, q.gx, k);
    qk.gy = __shfl_sync(0xffffffffu, q.gy, k);
    qk.h = __shfl_sync(0xffffffffu, q.h, k);
    qk.dcx = __shfl_sync(0xffffffffu, q.dcx, k);
    qk.dcy = __shfl_sync(0xffffffffu, q.dcy, k);
    qk.ex = __shfl_sync(0xffffffffu, q.ex, k);
    qk.ey = __shfl_sync(0xffffffffu, q.ey, k);
    qk.rl2 = __shfl_sync(0xffffffffu, q.rl2, k);
    qk.inv_sxx = __shfl_sync(0xffffffffu, q.inv_sxx, k);
    qk.slope = __shfl_sync(0xffffffffu, q.slope, k);
    qk.ok = __shfl_sync(0xffffffffu, q.ok ? 1 : 0, k) != 0;
    const float4 ck = make_float4(__shfl_sync(0xffffffffu, cx, k), __shfl_sync(0xffffffffu, cy, k), 0.f, 0.f);
    const uint32_t slot = base + (uint32_t)qq;
    if (qq < total && slot < cap) {
      int a0 = sx0, a1 = sx1, c0 = 1, c1 = 0;
      if (qk.ok) row_ranges(qk, ck, ty, W, H, sx0, sx1, tshift, a0, a1, c0, c1);
      if (clip) {  // an ROI binning: only the masked part of each range
        clip_to_mask(clip, clip_tiles_x, clip_tiles_y, ty, a0, a1);
        clip_to_mask(clip, clip_tiles_x, clip_tiles_y, ty, c0, c1);
        if (a0 > a1) { a0 = c0; a1 = c1; c0 = 1; c1 = 0; }
      }
      // empty ranges are stored as [1, 0]
      if (a0 > a1) { a0 = 1; a1 = 0; }
      if (c0 > c1) { c0 = 1; c1 = 0; }
      spans[slot] = make_uint2((uint32_t)a0 | ((uint32_t)a1 << 16), (uint32_t)c0 | ((uint32_t)c1 << 16));
    }
  }
  }
}

// ---------------------------------------------------------------- compaction
// A surfel enters the depth sort when its bounding rectangle is not empty and,
// for an ROI binning, when that rectangle holds at least one ROI tile. The union
// variant (dominant eye of a parallel two-eye call) takes every surfel either
// eye bins.
struct VisibleLoad {
  const uint32_t *cnt;
  const uint32_t *cnt_other;  // union with the other eye's binned set, or null
  const ushort4 *rect;
  const uint32_t *sat;        // summed-area table of the ROI mask, or null
  int tiles_x;
  __device__ uint32_t operator()(uint32_t i) const {
    // the count and the rectangle are loaded together (one memory round trip)
    const bool mine = cnt[i] > 0u;
    const ushort4 rc = sat ? rect[i] : make_ushort4(0, 0, 0, 0);
    if (cnt_other) return (mine || cnt_other[i] > 0u) ? 1u : 0u;
    if (!mine) return 0u;
    if (!sat) return 1u;
    return sat_any(sat, tiles_x, rc.y, rc.w, rc.x, rc.z) ? 1u : 0u;
  }
};

// What the compaction's last CTA sets up for the rest of a binning: the binned
// count, cleared row-span, list and tile-list counters, the chunks holding
// binned surfels and the size of the (tile, chunk) table scan over them.
struct BinCounts {
  uint32_t *n_out, *n_rows, *n_band, *n_items, *n_chunks, *n_table;  // n_rows may be null
  uint32_t chunk, ntiles;
  __device__ void set(uint32_t total) const {
    *n_out = total;
    if (n_rows) *n_rows = 0u;  // null: the spans are computed on another stream
    *n_band = 0u;
    *n_items = 0u;
    // at least one chunk, so that every tile's range is written
    const uint32_t nc = total > 0u ? (total + chunk - 1) / chunk : 1u;
    *n_chunks = nc;
    *n_table = nc * ntiles;
  }
};

struct CompactApply {
  const uint32_t *zkey;
  uint32_t *key_out, *val_out;
  BinCounts bc;
  using Payload = uint32_t;  // the depth key
  __device__ Payload fetch(uint32_t i, uint32_t v) const { return v ? zkey[i] : 0u; }
  __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t v, Payload key) const {
    if (v) {
      key_out[prefix] = key;
      val_out[prefix] = i;
    }
  }
  __device__ void end(uint32_t, uint32_t total) const { bc.set(total); }
};

// The affiliated eye's surfels in the dominant eye's depth order: a stable filter
// of that order. For a parallel rig both eyes' keys are identical, so the
// filtered order is exactly the affiliated (depth, index) order.
struct ReuseLoad {
  const uint32_t *uval, *n_union;
  uint32_t n_max;
  const uint32_t *cnt;   // this eye's tile counts
  const ushort4 *rect;
  const uint32_t *sat;   // summed-area table of the ROI mask, or null
  int tiles_x;
  __device__ uint32_t operator()(uint32_t i) const {
    if (i >= load_n(n_union, n_max)) return 0u;
    const uint32_t id = uval[i];
    // the count and the rectangle are loaded together (one memory round trip)
    const uint32_t c = cnt[id];
    const ushort4 rc = sat ? rect[id] : make_ushort4(0, 0, 0, 0);
    if (c == 0u) return 0u;
    if (!sat) return 1u;
    return sat_any(sat, tiles_x, rc.y, rc.w, rc.x, rc.z) ? 1u : 0u;
  }
};

struct ReuseApply {
  const uint32_t *uval, *zkey;
  uint32_t *key_out, *val_out;
  BinCounts bc;
  using Payload = uint2;  // surfel id, depth key
  __device__ Payload fetch(uint32_t i, uint32_t v) const {
    if (!v) return make_uint2(0u, 0u);
    const uint32_t id = uval[i];
    return make_uint2(id, zkey[id]);
  }
  __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t v, Payload p) const {
    if (v) {
      key_out[prefix] = p.y;
      val_out[prefix] = p.x;
    }
  }
  __device__ void end(uint32_t, uint32_t total) const { bc.set(total); }
};

// Keeps the dominant eye's depth order of the union for the affiliated eye.
__global__ void keep_union_kernel(const uint32_t *__restrict__ src, const uint32_t *__restrict__ n_ptr, uint32_t n_max,
                                  uint32_t *__restrict__ dst, uint32_t *__restrict__ n_union) {
  griddep_wait();
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_union = n;
}

// ---------------------------------------------------------------- counting sort by tile
//
// The depth-ordered surfels are cut into chunks of kBinWarps sub-chunks of
// `warp_surfels` consecutive surfels (one per warp) and the tile rows into bands
// of kBandRows.
//
//   band lists (one CTA per chunk): every warp lists, per band, the surfels of
//     its sub-chunk that reach the band (in depth order) with the span slot and
//     rows of their band part;
//   mode 0 (CTA per (chunk, band)): each warp counts its list's hits per tile;
//     the 8 counts of a (tile, chunk) go to table[tile][chunk] as 8 x 16 bits;
//   (a tile-major scan of the per-(tile, chunk) sums gives offs[tile][chunk],
//    where chunk c's run of the tile starts; offs[tile][0] starts the tile's list)
//   mode 1: each warp starts at offs[tile][c] plus the counts of the warps before
//     it and writes every surfel id to its slot.
//
// In modes 0 and 1 every warp keeps private per-tile counters for the band in
// shared memory and walks its list's instances 32 at a time, one (surfel, tile)
// per lane: a warp scan over the entries' instance counts (read from the row
// spans) gives each lane its entry, row and tile, so no lane loops over a span
// while others idle. The lanes of one step hold instances in depth order;
// lanes that reach the same tile are ranked by a per-tile bit mask of lanes, so
// every tile's list comes out in depth order. Both modes run the same walk code
// in one kernel, so the counts of mode 0 and the slots written in mode 1 always
// agree.
constexpr int kBinWarps = 8;
constexpr int kBinThreads = kBinWarps * 32;
constexpr int kBandRows = 4;
constexpr int kMaxBands = 256;  // tile rows <= kMaxBands * kBandRows = 1024 (8192 pixels at tile edge 8)

// One (surfel, band) entry: surfel id, span slot of its first row in the band,
// first row << 4 | rows in the band (1..kBandRows).
struct BandEntry {
  uint32_t id, sp, rows;
};
static_assert(sizeof(BandEntry) == kBandEntryBytes, "band entry layout");

struct BandArgs {
  const uint32_t *ids;     // depth-ordered binned surfels
  const uint32_t *n_vis;
  uint32_t n_max;
  const uint32_t *cnt;     // this eye's rectangle tile counts (0: not binned by this eye)
  const ushort4 *rect;
  const uint32_t *row_off;
  const uint32_t *sat;     // ROI mask summed-area table, or null
  int tiles_x, tiles_y;
  uint32_t warp_surfels;
  BandEntry *pool;         // all lists
  uint32_t pool_cap;
  uint32_t *pool_n;        // entries taken (device counter)
  uint2 *lists;            // [chunk][band][warp]: (first entry, entries)
  uint32_t *status;
};

// Band lists: one CTA of kBinWarps warps per sub-chunk (the surfels of one
// bin_kernel warp). The sub-chunk's 32-surfel groups are split into kBinWarps
// consecutive ranges, one per warp. Pass 0 counts each warp's (surfel, band)
// entries per band; a CTA-wide scan turns the counts into the band lists'
// places (bands in order, warps in order inside a band, so every list stays in
// depth order) with one pool reservation per sub-chunk; pass 1 walks the same
// groups again and writes the entries.
__global__ void __launch_bounds__(kBinThreads) band_list_kernel(BandArgs a) {
  griddep_wait();
  __shared__ uint32_t s_cnt[kBinWarps][kMaxBands];  // pass 0 counts, then each warp's write position
  __shared__ uint32_t s_scan[32];
  __shared__ uint32_t s_base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t nv = load_n(a.n_vis, a.n_max);
  const uint32_t sub = blockIdx.x;                  // sub-chunk: chunk sub / kBinWarps, warp sub % kBinWarps
  const uint32_t c = sub / kBinWarps;
  if (c * kBinWarps * a.warp_surfels >= nv) return;  // bin_kernel skips the whole chunk
  const int nb = (a.tiles_y + kBandRows - 1) / kBandRows;
  uint2 *my_lists = a.lists + ((size_t)c * nb) * kBinWarps + (sub % kBinWarps);  // stride kBinWarps per band
  const uint32_t s0 = sub * a.warp_surfels;
  const uint32_t s1 = min(s0 + a.warp_surfels, nv);
  // this warp's groups of 32 surfels: [g0, g1) of the sub-chunk's ng groups
  const uint32_t ng = s1 > s0 ? (s1 - s0 + 31) / 32 : 0u;
  const uint32_t g0 = ng * (uint32_t)w / kBinWarps, g1 = ng * (uint32_t)(w + 1) / kBinWarps;
  uint32_t *cnt = s_cnt[w];
  for (int b = lane; b < nb; b += 32) cnt[b] = 0u;
  __syncwarp();
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      // per band: the warps' exclusive offsets inside the band and the band's
      // total; then the bands' places in the sub-chunk's pool range
      __syncthreads();
      uint32_t tot = 0;
      static_assert(kMaxBands <= kBinThreads, "one thread per band");
      if (threadIdx.x < nb) {
        const int b = threadIdx.x;
#pragma unroll
        for (int ww = 0; ww < kBinWarps; ++ww) {
          const uint32_t v = s_cnt[ww][b];
          s_cnt[ww][b] = tot;
          tot += v;
        }
      }
      uint32_t band_off;
      const uint32_t all = block_exclusive_scan<kBinThreads>(threadIdx.x < nb ? tot : 0u, &band_off, s_scan);
      if (threadIdx.x == 0) {
        uint32_t base = 0;
        if (all > 0) base = atomicAdd(a.pool_n, all);
        if (all > 0 && (uint64_t)base + all > a.pool_cap) atomicOr(a.status, kStCapacity);
        s_base = base;
      }
      __syncthreads();
      if (threadIdx.x < nb) {
        const int b = threadIdx.x;
        const uint32_t at = s_base + band_off;
        const uint32_t keep = at >= a.pool_cap ? 0u : min(tot, a.pool_cap - at);
        my_lists[(size_t)b * kBinWarps] = make_uint2(at, keep);
#pragma unroll
        for (int ww = 0; ww < kBinWarps; ++ww) s_cnt[ww][b] += at;
      }
      __syncthreads();
    }
    for (uint32_t g = g0; g < g1; ++g) {  // warp-uniform
      const uint32_t j = s0 + g * 32u + (uint32_t)lane;
      int b0 = 1, b1 = 0, y0 = 0, y1 = -1, x0 = 0, x1 = -1;
      uint32_t id = 0, ro = 0;
      if (j < s1) id = a.ids[j];
      if (j < s1 && a.cnt[id] > 0u) {
        const ushort4 rc = a.rect[id];
        y0 = rc.y; y1 = rc.w; x0 = rc.x; x1 = rc.z;
        b0 = y0 / kBandRows;
        b1 = y1 / kBandRows;
        if (pass == 1) ro = a.row_off[id];
      }
      int bmin = b0 <= b1 ? b0 : 0x7fffffff, bmax = b0 <= b1 ? b1 : -1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
        bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
      }
      for (int b = bmin; b <= bmax; ++b) {  // warp-uniform
        const int lo = max(y0, b * kBandRows), hi = min(y1, b * kBandRows + kBandRows - 1);
        bool in = b >= b0 && b <= b1 && lo <= hi;
        if (in && a.sat) in = sat_any(a.sat, a.tiles_x, lo, hi, x0, x1);
        const uint32_t ball = __ballot_sync(0xffffffffu, in);
        if (pass == 1) {
          const uint32_t at = cnt[b] + (uint32_t)__popc(ball & lt);
          if (in && at < a.pool_cap)
            a.pool[at] = BandEntry{id, ro + (uint32_t)(lo - y0), ((uint32_t)lo << 4) | (uint32_t)(hi - lo + 1)};
        }
        __syncwarp();
        if (lane == 0) cnt[b] += (uint32_t)__popc(ball);
        __syncwarp();
      }
    }
  }
}

struct BinArgs {
  const uint32_t *n_vis;   // binned surfels (device)
  uint32_t n_max;
  const BandEntry *pool;
  const uint2 *lists;      // [chunk][band][warp]
  const uint2 *spans;      // tile ranges of every rectangle row (rows_kernel)
  uint32_t span_cap;
  const uint8_t *mask;     // ROI tile mask, or null
  int tiles_x, tiles_y;
  uint32_t warp_surfels;   // surfels per warp sub-chunk (< 65536)
  uint32_t nch;            // chunks (row length of the tables)
  uint4 *table;            // [tile][chunk] 8 x 16-bit per-warp counts
  const uint32_t *offs;    // [tile][chunk] exclusive offsets (mode 1)
  uint32_t cap;            // instance capacity
  uint32_t *ival;          // surfel id per instance
  uint32_t *ikey;          // tile id per instance, or null
  uint32_t *cnt_bin;       // tiles per surfel, or null (mode 0)
};

__device__ __forceinline__ int shi(int v, int k) { return __shfl_sync(0xffffffffu, v, k); }

__device__ __forceinline__ uint32_t half16(const uint4 &v, int w) {
  const uint32_t x = w < 2 ? v.x : w < 4 ? v.y : w < 6 ? v.z : v.w;
  return (w & 1) ? x >> 16 : x & 0xffffu;
}

// Six resident CTAs per SM (40 registers, no spills): the walk is bound by the
// latency of its shuffles, gathers and shared-memory atomics, and the extra
// warps cover it (four CTAs took 56 registers and measured slower).
__global__ void __launch_bounds__(kBinThreads, 6) bin_kernel(BinArgs a, int mode) {
  griddep_wait();
  extern __shared__ uint32_t s_dyn[];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t nv = load_n(a.n_vis, a.n_max);
  const uint32_t c = blockIdx.x;
  if (c * kBinWarps * a.warp_surfels >= nv) return;  // the scan reads these counts as 0
  const int tx_n = a.tiles_x;
  const int nb = (a.tiles_y + kBandRows - 1) / kBandRows;
  const int by0 = (int)blockIdx.y * kBandRows;
  const int by1 = min(by0 + kBandRows, a.tiles_y) - 1;
  const int BT = (by1 - by0 + 1) * tx_n;
  const int BTmax = kBandRows * tx_n;
  uint32_t *s_cnt = s_dyn;                      // [kBinWarps][BTmax]
  uint32_t *s_msk = s_dyn + kBinWarps * BTmax;  // [kBinWarps][BTmax], mode 1
  const size_t t0 = (size_t)by0 * tx_n;         // first tile of the band
  const uint2 *lists = a.lists + ((size_t)c * nb + blockIdx.y) * kBinWarps;
  if (!__syncthreads_or(tid < kBinWarps && lists[tid].y > 0u)) {  // nothing reaches the band
    if (mode == 0)
      for (int bt = tid; bt < BT; bt += kBinThreads) a.table[(t0 + bt) * a.nch + c] = make_uint4(0, 0, 0, 0);
    return;
  }
  if (mode == 0) {
    for (int i = tid; i < kBinWarps * BTmax; i += kBinThreads) s_dyn[i] = 0u;
  } else {  // each warp's first slot per tile; masks cleared
    for (int bt = tid; bt < BT; bt += kBinThreads) {
      const size_t e = (t0 + bt) * a.nch + c;
      const uint4 v = a.table[e];
      uint32_t base = a.offs[e];
#pragma unroll
      for (int ww = 0; ww < kBinWarps; ++ww) {
        s_cnt[ww * BTmax + bt] = base;
        s_msk[ww * BTmax + bt] = 0u;
        base += half16(v, ww);
      }
    }
  }
  __syncthreads();
  uint32_t *my_cnt = s_cnt + w * BTmax;
  uint32_t *my_msk = s_msk + w * BTmax;
  const uint2 li = lists[w];
  const BandEntry *q = a.pool + li.x;
  const int qn = (int)li.y;
  // All loops below are warp-uniform. A step loads 32 entries (one per lane)
  // and the instance counts of their rows from the row spans; a warp scan of
  // those counts then maps instance g of the step to its entry, row and tile,
  // and the step's instances are taken 32 at a time, one per lane, so no lane
  // loops over a span while others idle.
  for (int qpos = 0; qpos < qn; qpos += 32) {
    const int e = qpos + lane;
    uint32_t id = 0, sp = 0;
    int lo = 0;
    int rc[kBandRows];  // instances per row of the entry
    int pk[kBandRows];  // the row's ranges: a0 | na << 10 | c0 << 20 (na = a1 - a0 + 1 or 0)
#pragma unroll
    for (int r = 0; r < kBandRows; ++r) rc[r] = pk[r] = 0;
    if (e < qn) {
      const BandEntry en = q[e];
      id = en.id;
      sp = en.sp;
      lo = (int)(en.rows >> 4);
      const int nr = (int)(en.rows & 15u);
#pragma unroll
      for (int r = 0; r < kBandRows; ++r) {
        if (r < nr && sp + (uint32_t)r < a.span_cap) {
          const uint2 v = a.spans[sp + (uint32_t)r];
          const int a0 = (int)(v.x & 0xffffu), a1 = (int)(v.x >> 16);
          const int c0 = (int)(v.y & 0xffffu), c1 = (int)(v.y >> 16);
          const int na = max(a1 - a0 + 1, 0);
          rc[r] = na + max(c1 - c0 + 1, 0);
          pk[r] = (a0 & 1023) | (na << 10) | ((c0 & 1023) << 20);
        }
      }
    }
    int nt = 0;
#pragma unroll
    for (int r = 0; r < kBandRows; ++r) nt += rc[r];
    int incl = nt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = shi(incl, 31);
    for (int g0 = 0; g0 < total; g0 += 32) {
      const int g = g0 + lane;
      const bool act = g < total;
      int kl = 0, kh = 31;  // entry of instance g: first lane whose inclusive prefix exceeds it
#pragma unroll
      for (int it = 0; it < 5; ++it) {
        const int mid = (kl + kh) >> 1;
        if (shi(incl, mid) > g) kh = mid; else kl = mid + 1;
      }
      const int k = kl;
      const uint32_t sid = (uint32_t)shi((int)id, k);
      // index of the instance among entry k's instances, then its row r and
      // the row's ranges (all from lane k's registers: independent shuffles)
      int t = g - (shi(incl, k) - shi(nt, k));
      int rcs[kBandRows], pks[kBandRows];
#pragma unroll
      for (int rr = 0; rr < kBandRows; ++rr) {
        rcs[rr] = shi(rc[rr], k);
        pks[rr] = shi(pk[rr], k);
      }
      int r = 0, w = pks[0];
#pragma unroll
      for (int rr = 0; rr < kBandRows - 1; ++rr) {
        if (r == rr && t >= rcs[rr]) {
          t -= rcs[rr];
          r = rr + 1;
          w = pks[rr + 1];
        }
      }
      const int ty = shi(lo, k) + r;
      // the lane's tile: the t-th of the row's ranges [a0, a1] u [c0, c1]
      const int a0 = w & 1023, na = (w >> 10) & 1023, c0 = (w >> 20) & 1023;
      const int tx = t < na ? a0 + t : c0 + (t - na);
      const bool valid = act && (!a.mask || a.mask[(size_t)ty * tx_n + tx] != 0);
      const int bt = (ty - by0) * tx_n + tx;
      if (mode == 0) {
        if (valid) {
          atomicAdd(&my_cnt[bt], 1u);
          if (a.cnt_bin) atomicAdd(&a.cnt_bin[sid], 1u);
        }
      } else {
        // lanes on one tile are ranked by lane (depth order); the highest of
        // them advances the tile's counter
        if (valid) atomicOr(&my_msk[bt], 1u << lane);
        __syncwarp();
        uint32_t m = 0, base = 0;
        if (valid) {
          m = my_msk[bt];
          base = my_cnt[bt];
          const uint32_t pos = base + (uint32_t)__popc(m & lt);
          if (pos < a.cap) {
            a.ival[pos] = sid;
            if (a.ikey) a.ikey[pos] = (uint32_t)(ty * tx_n + tx);
          }
        }
        __syncwarp();
        if (valid && lane == 31 - __clz(m)) {
          my_cnt[bt] = base + (uint32_t)__popc(m);
          my_msk[bt] = 0u;
        }
        __syncwarp();
      }
    }
  }
  if (mode == 0) {
    __syncthreads();
    for (int bt = tid; bt < BT; bt += kBinThreads) {
      uint32_t h[kBinWarps];
#pragma unroll
      for (int ww = 0; ww < kBinWarps; ++ww) h[ww] = s_cnt[ww * BTmax + bt];
      a.table[(t0 + bt) * a.nch + c] =
          make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
    }
  }
}

// The tile-major scan runs over the (tile, chunk) entries of the chunks that
// hold binned surfels only (one chunk when none does): element i is tile
// i / n_chunks, chunk i % n_chunks (the table rows keep their full length nch).
struct BinTableLoad {
  const uint4 *table;
  const uint32_t *n_chunks, *n_vis;
  uint32_t nch, chunk;
  __device__ uint32_t operator()(uint32_t i) const {
    const uint32_t na = *n_chunks, c = i % na;
    if (c * chunk >= *n_vis) return 0u;  // only with no binned surfel: bin_kernel wrote nothing
    const uint4 v = table[(size_t)(i / na) * nch + c];
    const uint32_t lo = (v.x & 0xffffu) + (v.y & 0xffffu) + (v.z & 0xffffu) + (v.w & 0xffffu);
    return lo + (v.x >> 16) + (v.y >> 16) + (v.z >> 16) + (v.w >> 16);
  }
};

// Offsets of every (tile, chunk) run; the first chunk's entry of a tile also
// gives the tile's range (its start, and the end of the tile before it), and a
// masked binning lists its masked tiles for the persistent rasterizer (in any
// order: the rasterizer's tiles are independent).
struct BinOffsetApply {
  uint32_t *offs;
  const uint32_t *n_chunks;
  uint32_t nch;
  uint32_t *n_inst, *n_sort;
  uint32_t cap;
  uint32_t *status;
  uint2 *ranges;
  int ntiles;
  const uint8_t *mask;  // null for a full binning
  uint32_t *items, *n_items;
  using Payload = uint2;  // chunks in use, the tile's mask byte (first chunk only)
  __device__ Payload fetch(uint32_t i, uint32_t) const {
    const uint32_t na = *n_chunks;
    return make_uint2(na, (mask && i % na == 0u) ? (uint32_t)mask[i / na] : 0u);
  }
  __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t, Payload pl) const {
    const uint32_t na = pl.x;
    const uint32_t t = i / na, c = i % na;
    offs[(size_t)t * nch + c] = prefix;
    if (c != 0u) return;
    const uint32_t p = min(prefix, cap);
    ranges[t].x = p;
    if (t > 0u) ranges[t - 1].y = p;
    if (pl.y) items[atomicAdd(n_items, 1u)] = t;
  }
  __device__ void end(uint32_t, uint32_t total) const {
    *n_inst = total;
    *n_sort = total < cap ? total : cap;
    if (total > cap) atomicOr(status, kStCapacity);
    if (ntiles > 0) ranges[ntiles - 1].y = min(total, cap);
  }
};

uint32_t bin_warp_surfels(int max_surfels) {
  const uint32_t per = ((uint32_t)max_surfels + kBinWarps * 256 - 1) / (kBinWarps * 256);
  uint32_t r = (per + 31) / 32 * 32;
  if (r < 64) r = 64;
  if (r > 32768) r = 32768;  // per-warp counts are 16-bit
  return r;
}

size_t band_list_words(int max_surfels, int max_tiles_y) {
  return (size_t)bin_chunks(max_surfels) * ((max_tiles_y + kBandRows - 1) / kBandRows) * kBinWarps;
}

uint32_t bin_chunks(int max_surfels) {
  const uint32_t chunk = kBinWarps * bin_warp_surfels(max_surfels);
  const uint32_t n = ((uint32_t)max_surfels + chunk - 1) / chunk;
  return n < 1 ? 1 : n;
}

size_t bin_smem_bytes(int tiles_x) { return 2 * sizeof(uint32_t) * kBinWarps * kBandRows * (size_t)tiles_x; }

// The opt-in is a property of the kernel on the device, shared by every
// context: it only ever grows, so a small context created after a large one
// keeps the large one's limit.
cudaError_t prepare_binning(int max_tiles_x) {
  static std::mutex mu;
  static int granted[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int want = (int)bin_smem_bytes(max_tiles_x);
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && granted[dev] >= want) return cudaSuccess;
  e = cudaFuncSetAttribute(bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (e == cudaSuccess && dev >= 0 && dev < 64) granted[dev] = want;
  return e;
}

cudaError_t launch_binning(const Workspace &ws, int eye, int n, int tiles_x, int tiles_y,
                           const uint8_t *tile_mask, cudaStream_t s, int order, const uint8_t *roi16, int W,
                           int H, int tshift, const SideRows *rows) {
  const BinScratch &b = ws.bin[eye];
  cudaError_t err;
  Counters *ctr = ws.ctr;
  const int ntiles = tiles_x * tiles_y;
  const uint32_t cap = (uint32_t)ws.max_inst[eye];
  const RadixScratch rs{b.rs_hist, b.rs_hist + kRsPasses * 256, b.rs_status, b.rs_ctl, &ctr->status};
  if (tile_mask) {  // (the rasterizer-grid mask and) its summed-area table
    launch_k(mask_sat_kernel, 1, 1024, 0, s, const_cast<uint8_t *>(tile_mask), tiles_x, tiles_y, b.mask_sat, roi16,
             (W + kTile - 1) / kTile, (H + kTile - 1) / kTile, roi16 ? tshift : 4, b.mask_clip,
             roi16 ? b.items16 : nullptr);
    GS_LAUNCHED(1);
  }
  // the row spans need only the preprocessed records (and an ROI binning's mask
  // tables): on a second stream they run beside the compaction and the sort.
  // Beside a depth sort a small grid leaves those latency-bound kernels their
  // SMs; beside the filter scan alone (the kept dominant order) the spans are
  // the longer branch and take a fuller grid
  const bool side_rows = rows && n > 0;
  if (side_rows) {
    const bool reuse = order == kOrderReuse;  // the candidates: the kept dominant order, else every surfel
    const int cap_g = sm_grid_cap(reuse ? 6 : 2);
    const int grid = cap_g < (n + 255) / 256 ? cap_g : (n + 255) / 256;
    err = cudaEventRecord(rows->fork, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(rows->stream, rows->fork, 0);
    if (err == cudaSuccess) err = cudaMemsetAsync(&ctr->n_rows[eye], 0, sizeof(uint32_t), rows->stream);
    if (err == cudaSuccess)
      err = launch_k(rows_kernel, grid, 256, 0, rows->stream, reuse ? ws.uval : nullptr,
                     reuse ? &ctr->n_union : nullptr, (uint32_t)n, ws.rec[eye], ws.rect[eye], ws.cnt[eye], ws.cams,
                     eye, ws.prim, ws.row_off[eye], ws.spans[eye], cap, &ctr->n_rows[eye], &ctr->status,
                     tile_mask ? b.mask_clip : nullptr, tiles_x, tiles_y, tile_mask ? b.mask_sat : nullptr);
    GS_LAUNCHED(1);
    if (err == cudaSuccess) err = cudaEventRecord(rows->join, rows->stream);
    if (err != cudaSuccess) return err;
  }
  const uint32_t chunk = kBinWarps * ws.bin_warp_surfels;
  const BinCounts bc{&ctr->n_vis[eye], side_rows ? nullptr : &ctr->n_rows[eye], &ctr->n_band[eye],
                     &ctr->n_items[eye], &ctr->n_chunks[eye], &ctr->n_table[eye], chunk, (uint32_t)ntiles};
  // 1. compact the binned surfels: (depth bits, surfel id)
  const uint32_t *sat = tile_mask ? b.mask_sat : nullptr;
  if (order == kOrderReuse) {  // the dominant order, filtered: already depth-ordered
    err = scan_launch(ReuseLoad{ws.uval, &ctr->n_union, (uint32_t)n, ws.cnt[eye], ws.rect[eye], sat, tiles_x},
                      ReuseApply{ws.uval, ws.zkey[eye], b.dkey[0], b.dval[0], bc},
                      (const uint32_t *)nullptr, (uint32_t)n, b.scan_tiles, b.scan_ticket, &ctr->status, s);
  } else {
    err = scan_launch(VisibleLoad{ws.cnt[eye], order == kOrderUnion ? ws.cnt[1 - eye] : nullptr, ws.rect[eye], sat,
                                  tiles_x},
                      CompactApply{ws.zkey[eye], b.dkey[0], b.dval[0], bc},
                      (const uint32_t *)nullptr, (uint32_t)n, b.scan_tiles, b.scan_ticket, &ctr->status, s);
  }
  if (err != cudaSuccess) return err;
  // 2. tile ranges of every rectangle row of those surfels (n_rows and n_band
  // were cleared by the compaction)
  if (n > 0 && !side_rows) {
    launch_k(rows_kernel, (n + 255) / 256, 256, 0, s, b.dval[0], &ctr->n_vis[eye], (uint32_t)n, ws.rec[eye],
                                                ws.rect[eye], ws.cnt[eye], ws.cams, eye, ws.prim, ws.row_off[eye],
                                                ws.spans[eye], cap, &ctr->n_rows[eye],
                                                &ctr->status, tile_mask ? b.mask_clip : nullptr, tiles_x, tiles_y,
                                                (const uint32_t *)nullptr);
    GS_LAUNCHED(1);
  }
  // 3. depth order (the low 32 bits of the packed key; stable, so ties keep id order)
  int which = 0;
  if (order != kOrderReuse &&
      (err = radix_sort(b.dkey, b.dval, &ctr->n_vis[eye], (uint32_t)n, 32, rs, &which, s)) != cudaSuccess)
    return err;
  if (order == kOrderUnion && n > 0) {  // kept for the affiliated eye
    const int cap = sm_grid_cap(8);
    const int g = (int)((n + 255) / 256 < cap ? (n + 255) / 256 : cap);
    if ((err = launch_k(keep_union_kernel, g, 256, 0, s, b.dval[which], &ctr->n_vis[eye], (uint32_t)n, ws.uval,
                        &ctr->n_union)) != cudaSuccess)
      return err;
    GS_LAUNCHED(1);
  }
  const int nbands = (tiles_y + kBandRows - 1) / kBandRows;
  if (side_rows && (err = cudaStreamWaitEvent(s, rows->join, 0)) != cudaSuccess) return err;
  // 4. per chunk: each warp's depth-ordered (surfel, band) lists
  BandArgs ba;
  ba.ids = b.dval[which];
  ba.n_vis = &ctr->n_vis[eye];
  ba.n_max = (uint32_t)n;
  ba.cnt = ws.cnt[eye];
  ba.rect = ws.rect[eye];
  ba.row_off = ws.row_off[eye];
  ba.sat = tile_mask ? b.mask_sat : nullptr;
  ba.tiles_x = tiles_x;
  ba.tiles_y = tiles_y;
  ba.warp_surfels = ws.bin_warp_surfels;
  ba.pool = b.band_pool;
  ba.pool_cap = ws.band_pool_cap[eye];
  ba.pool_n = &ctr->n_band[eye];
  ba.lists = b.band_lists;
  ba.status = &ctr->status;
  launch_k(band_list_kernel, ws.bin_nch * kBinWarps, kBinThreads, 0, s, ba);
  GS_LAUNCHED(1);
  BinArgs a;
  a.n_vis = &ctr->n_vis[eye];
  a.n_max = (uint32_t)n;
  a.pool = b.band_pool;
  a.lists = b.band_lists;
  a.spans = ws.spans[eye];
  a.span_cap = cap;
  a.mask = tile_mask;
  a.tiles_x = tiles_x;
  a.tiles_y = tiles_y;
  a.warp_surfels = ws.bin_warp_surfels;
  a.nch = ws.bin_nch;
  a.table = b.bin_table;
  a.offs = b.bin_offs;
  a.cap = cap;
  a.ival = b.ival;
  a.ikey = ws.keep_intermediates ? b.ikey : nullptr;
  a.cnt_bin = ws.keep_intermediates ? ws.cnt_bin : nullptr;
  if (a.cnt_bin && n > 0 && (err = cudaMemsetAsync(a.cnt_bin, 0, sizeof(uint32_t) * (size_t)n, s)) != cudaSuccess)
    return err;
  const dim3 grid(ws.bin_nch, (unsigned)nbands);
  // 5. per-warp counts per (tile, chunk)
  launch_k(bin_kernel, grid, kBinThreads, bin_smem_bytes(tiles_x) / 2, s, a, 0);
  GS_LAUNCHED(1);
  // 6. tile-major scan over the chunks that hold binned surfels: where every
  // (tile, chunk) run starts, every tile's range and, for a mask, the tile list
  err = scan_launch(BinTableLoad{b.bin_table, &ctr->n_chunks[eye], &ctr->n_vis[eye], ws.bin_nch, chunk},
                    BinOffsetApply{b.bin_offs, &ctr->n_chunks[eye], ws.bin_nch, &ctr->n_inst[eye], &ctr->n_sort[eye],
                                   cap, &ctr->status, b.ranges, ntiles, tile_mask, b.items, &ctr->n_items[eye]},
                    &ctr->n_table[eye], (uint32_t)ntiles * ws.bin_nch, b.scan_tiles, b.scan_ticket, &ctr->status, s);
  if (err != cudaSuccess) return err;
  // 7. every surfel id to its slot
  launch_k(bin_kernel, grid, kBinThreads, bin_smem_bytes(tiles_x), s, a, 1);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace gs
