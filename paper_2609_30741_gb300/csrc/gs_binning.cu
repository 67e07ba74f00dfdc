// Tile binning: an on-device LSD radix sort of packed (tile id | depth) keys.
//
// Paper: Sec. 3.1 Stage 1 and Sec. 3.5 (16x16 tiles of the 2DGS/3DGS tile
// rasterizer; Sec. 2.2 keeps its depth ordering).
//
// The sort key of an instance is (tile id << 32) | float_bits(z_c). Every
// instance of a surfel shares the depth digits, so the LSD passes over the low
// 32 bits are run on the visible surfels *before* they are duplicated into
// instances, and only the tile digits are sorted per instance. Because LSD
// passes are stable, this yields exactly the order of a full 64-bit LSD sort of
// the packed keys (ties broken by surfel index), with far less data moved.
//
// Pipeline per eye (all counts stay on the device):
//   1. compact the surfels with a non-zero tile count (scan) -> (depth bits, id)
//   2. 4 radix passes over the depth bits
//   3. scan of the tile counts in depth order -> instance offsets
//   4. emit (tile id, surfel id) for every touched tile (restricted to the ROI
//      tile mask when one is given)
//   5. 1-2 radix passes over the tile ids (stable: depth order kept per tile)
//   6. [start, end) range of every tile
#include "gs_internal.cuh"
#include "gs_scan.cuh"

namespace gs {

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

// Tile count of a surfel restricted to the tiles set in `mask`.
__global__ void roi_count_kernel(const ushort4 *__restrict__ rect, const uint32_t *__restrict__ cnt,
                                 const uint8_t *__restrict__ mask, int tiles_x, int n,
                                 uint32_t *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c = 0;
  if (cnt[i]) {
    const ushort4 r = rect[i];
    for (int ty = r.y; ty <= r.w; ++ty)
      for (int tx = r.x; tx <= r.z; ++tx) c += mask[ty * tiles_x + tx] ? 1u : 0u;
  }
  out[i] = c;
}

// One thread per depth-sorted surfel writes its (tile, surfel) instances.
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
                                                   const uint32_t *__restrict__ cnt,
                                                   const ushort4 *__restrict__ rect,
                                                   const uint8_t *__restrict__ mask, int tiles_x,
                                                   const uint32_t *__restrict__ n_vis, uint32_t cap,
                                                   uint32_t *__restrict__ ikey, uint32_t *__restrict__ ival) {
  const uint32_t n = *n_vis;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t id = ids[j];
    const uint32_t base = offs[j];
    const uint32_t c = cnt[id];
    if ((uint64_t)base + c > cap) continue;  // capacity exceeded: flagged by the offset scan
    const ushort4 r = rect[id];
    uint32_t k = base;
    for (int ty = r.y; ty <= r.w; ++ty) {
      for (int tx = r.x; tx <= r.z; ++tx) {
        const uint32_t t = (uint32_t)(ty * tiles_x + tx);
        if (mask && !mask[t]) continue;
        ikey[k] = t;
        ival[k] = id;
        ++k;
      }
    }
  }
}

__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ n_ptr,
                                                     uint2 *__restrict__ ranges) {
  const uint32_t n = *n_ptr;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
  }
}

static int bits_for(int ntiles) {
  int b = 0;
  while ((1 << b) < ntiles) ++b;
  return b < 1 ? 1 : b;
}

cudaError_t launch_binning(const Workspace &ws, int eye, int n, int tiles_x, int tiles_y,
                           const uint8_t *tile_mask, cudaStream_t s) {
  cudaError_t err;
  Counters *ctr = ws.ctr;
  const int ntiles = tiles_x * tiles_y;
  const uint32_t *cnt = ws.cnt[eye];
  if (tile_mask) {
    if (n > 0) {
      roi_count_kernel<<<(n + 255) / 256, 256, 0, s>>>(ws.rect[eye], ws.cnt[eye], tile_mask, tiles_x, n, ws.cnt_roi);
      GS_LAUNCHED(1);
    }
    cnt = ws.cnt_roi;
  }
  if ((err = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * (size_t)ntiles, s)) != cudaSuccess) return err;
  // 1. compact the binned surfels: (depth bits, surfel id)
  err = scan_launch(FlagLoad{cnt}, CompactApply{ws.zkey[eye], ws.dkey[0], ws.dval[0], &ctr->n_vis[eye]},
                    (const uint32_t *)nullptr, (uint32_t)n, ws.scan_sums, nullptr, s);
  if (err != cudaSuccess) return err;
  // 2. depth digits (the low 32 bits of the packed key)
  int which = 0;
  if ((err = radix_sort(ws.dkey, ws.dval, &ctr->n_vis[eye], (uint32_t)n, 32, ws.hist, &which, s)) != cudaSuccess)
    return err;
  const uint32_t *ids = ws.dval[which];
  // 3. instance offsets in depth order
  const uint32_t cap = (uint32_t)ws.max_instances;
  err = scan_launch(SortedCountLoad{cnt, ids}, OffsetApply{ws.offs, &ctr->n_inst[eye], &ctr->n_sort[eye], cap, &ctr->status},
                    &ctr->n_vis[eye], (uint32_t)n, ws.scan_sums, nullptr, s);
  if (err != cudaSuccess) return err;
  // 4. emission
  const int emit_blocks = n > 0 ? min((n + 255) / 256, 152 * 8) : 1;
  emit_kernel<<<emit_blocks, 256, 0, s>>>(ids, ws.offs, cnt, ws.rect[eye], tile_mask, tiles_x, &ctr->n_vis[eye],
                                          cap, ws.ikey[0], ws.ival[0]);
  GS_LAUNCHED(1);
  // 5. tile digits (the high bits of the packed key)
  if ((err = radix_sort(ws.ikey, ws.ival, &ctr->n_sort[eye], cap, bits_for(ntiles), ws.hist, &which, s)) != cudaSuccess)
    return err;
  // 6. ranges
  ranges_kernel<<<152 * 8, 256, 0, s>>>(ws.ikey[which], &ctr->n_sort[eye], ws.ranges);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

// Buffer index holding the sorted instances: one pass per 8 tile bits, each pass
// flips between the two buffers.
int sorted_buffer(int ntiles) { return ((bits_for(ntiles) + 7) / 8) & 1; }

}  // namespace gs
