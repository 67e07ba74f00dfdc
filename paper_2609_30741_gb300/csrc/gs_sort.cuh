// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8 bits per pass,
// with a device-resident element count.
//
// Each pass has three phases with no waiting between CTAs:
//   1. every tile of 2048 pairs counts its digits into a [digit][tile] table;
//   2. one device-wide exclusive scan of that table in digit-major order gives,
//      for every (digit, tile), where the tile's run of that digit starts;
//   3. every tile ranks its pairs stably (per warp with bit ballots, then across
//      warps), sorts them locally in shared memory and writes each digit run to
//      its place with coalesced stores.
// Tiles are independent in phases 1 and 3, so the passes scale with the number
// of SMs instead of waiting on a chain of predecessor tiles.
#pragma once

#include "gs_internal.cuh"
#include "gs_launch.cuh"
#include "gs_scan.cuh"

namespace gs {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048 pairs per tile

// n_table = 256 * number of tiles, written by phase 1 for the scan of phase 2.
// With `offs` given (small tables), the last block to finish (counted on
// *ticket, which it resets) also runs phase 2: thread d scans digit d's row.
static __global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const uint32_t *__restrict__ keys,
                                                                     const uint32_t *n_ptr, uint32_t n_max, int shift,
                                                                     uint32_t *__restrict__ table,
                                                                     uint32_t *__restrict__ n_table,
                                                                     uint32_t *__restrict__ offs, uint32_t *ticket) {
  griddep_wait();
  __shared__ uint32_t h[kRsThreads / 32][256];
  __shared__ uint32_t s_last, s_scan[32];
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t ntiles = (n + kRsTile - 1) / kRsTile;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_table = 256u * ntiles;
  uint32_t(*hw) = h[threadIdx.x >> 5];
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int i = threadIdx.x; i < (kRsThreads / 32) * 256; i += kRsThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t base = t * (uint32_t)kRsTile;
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t i = base + (uint32_t)(j * kRsThreads + threadIdx.x);
      if (i < n) atomicAdd(&hw[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) c += h[w][threadIdx.x];
    table[(size_t)threadIdx.x * ntiles + t] = c;
    __syncthreads();
  }
  if (!offs) return;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const uint32_t *row = table + (size_t)threadIdx.x * ntiles;
  uint32_t tot = 0;
  for (uint32_t t = 0; t < ntiles; ++t) tot += __ldcg(row + t);
  uint32_t base;
  block_exclusive_scan<kRsThreads>(tot, &base, s_scan);
  uint32_t *orow = offs + (size_t)threadIdx.x * ntiles;
  for (uint32_t t = 0; t < ntiles; ++t) {
    const uint32_t v = __ldcg(row + t);
    orow[t] = base;
    base += v;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

struct TableLoad {
  const uint32_t *table;
  __device__ uint32_t operator()(uint32_t i) const { return table[i]; }
};

struct TableApply {
  uint32_t *offs;
  __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t) const { offs[i] = prefix; }
  __device__ void end(uint32_t, uint32_t) const {}
};

static __global__ void __launch_bounds__(kRsThreads, 4) rs_scatter_kernel(const uint32_t *__restrict__ kin,
                                                                           const uint32_t *__restrict__ vin,
                                                                           uint32_t *__restrict__ kout,
                                                                           uint32_t *__restrict__ vout,
                                                                           const uint32_t *n_ptr, uint32_t n_max,
                                                                           int shift,
                                                                           const uint32_t *__restrict__ offs) {
  griddep_wait();
  constexpr int NW = kRsThreads / 32;
  __shared__ uint32_t s_warp[NW][256];
  __shared__ uint32_t s_local_base[256], s_global[256];
  __shared__ uint32_t s_keys[kRsTile], s_vals[kRsTile];
  __shared__ uint32_t s_scan[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t ntiles = (n + kRsTile - 1) / kRsTile;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t base = t * (uint32_t)kRsTile;
    for (int i = tid; i < NW * 256; i += kRsThreads) (&s_warp[0][0])[i] = 0;
    s_global[tid] = offs[(size_t)tid * ntiles + t];
    __syncthreads();
    // warp w owns pairs [w * 32 * kRsItems, (w + 1) * 32 * kRsItems) of the tile
    uint32_t k[kRsItems], r[kRsItems], v[kRsItems];
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {  // values loaded with the keys: no second wait
      const uint32_t i = base + (uint32_t)(wid * 32 * kRsItems + j * 32 + lane);
      k[j] = i < n ? kin[i] : 0u;
      v[j] = i < n ? vin[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t i = base + (uint32_t)(wid * 32 * kRsItems + j * 32 + lane);
      const bool ok = i < n;
      const uint32_t d = (k[j] >> shift) & 255u;
      // lanes holding the same digit: intersect one ballot per digit bit
      uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bb = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bb : ~bb;
      }
      // the lowest such lane reserves the slots for the group in one shared atomic
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (ok && lane == leader) before = atomicAdd(&s_warp[wid][d], (uint32_t)__popc(peers));
      before = __shfl_sync(0xffffffffu, before, leader < 0 ? 0 : leader);
      r[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    // digit d = tid: the tile's count and each warp's offset inside the digit run
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = s_warp[w][tid];
      s_warp[w][tid] = cnt;
      cnt += c;
    }
    {
      uint32_t ex;
      block_exclusive_scan<kRsThreads>(cnt, &ex, s_scan);
      s_local_base[tid] = ex;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t i = base + (uint32_t)(wid * 32 * kRsItems + j * 32 + lane);
      if (i < n) {
        const uint32_t d = (k[j] >> shift) & 255u;
        const uint32_t pos = s_local_base[d] + s_warp[wid][d] + r[j];
        s_keys[pos] = k[j];
        s_vals[pos] = v[j];
      }
    }
    __syncthreads();
    const uint32_t tn = min((uint32_t)kRsTile, n - base);
    for (uint32_t i = tid; i < tn; i += kRsThreads) {
      const uint32_t key = s_keys[i];
      const uint32_t d = (key >> shift) & 255u;
      const uint32_t gp = s_global[d] + (i - s_local_base[d]);
      kout[gp] = key;
      vout[gp] = s_vals[i];
    }
    __syncthreads();
  }
}

struct RadixScratch {
  uint32_t *table;            // [256][tiles]
  uint32_t *offs;             // [256][tiles]
  uint32_t *n_table;          // one word
  unsigned long long *tiles;  // look-back words of the table scan
  uint32_t *ticket;           // scan control words (the first is 0 between scans)
  uint32_t *status;           // device status word
};

inline size_t radix_table_words(size_t n_max) { return 256 * ((n_max + kRsTile - 1) / kRsTile + 1); }

inline int radix_grid(uint32_t n_max) {
  const uint32_t tiles = (n_max + kRsTile - 1) / kRsTile;
  return (int)(tiles < 1 ? 1 : (tiles > 152 * 8 ? 152 * 8 : tiles));
}

// Sorts on bits [0, bits); the result lands in buffer index *which.
inline cudaError_t radix_sort(uint32_t *const keys[2], uint32_t *const vals[2], const uint32_t *n_ptr, uint32_t n_max,
                              int bits, const RadixScratch &sc, int *which, cudaStream_t s) {
  const int npass = (bits + 7) / 8;
  const int grid = radix_grid(n_max);
  const uint32_t table_max = (uint32_t)radix_table_words(n_max);
  // small tables (<= 32 tiles per digit row) are scanned by the histogram
  // kernel's last block: one launch fewer; larger rows scan faster in parallel
  const bool fused = (n_max + kRsTile - 1) / kRsTile <= 32;
  int cur = 0;
  for (int p = 0; p < npass; ++p) {
    launch_k(rs_hist_kernel, grid, kRsThreads, 0, s, keys[cur], n_ptr, n_max, 8 * p, sc.table, sc.n_table,
                                               fused ? sc.offs : nullptr, sc.ticket);
    GS_LAUNCHED(1);
    if (!fused) {
      cudaError_t e = scan_launch(TableLoad{sc.table}, TableApply{sc.offs}, sc.n_table, table_max, sc.tiles,
                                  sc.ticket, sc.status, s);
      if (e != cudaSuccess) return e;
    }
    launch_k(rs_scatter_kernel, grid, kRsThreads, 0, s, keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_ptr, n_max,
                                                  8 * p, sc.offs);
    GS_LAUNCHED(1);
    cur ^= 1;
  }
  *which = cur;
  return cudaGetLastError();
}

}  // namespace gs
