// Device-wide exclusive scan and LSD radix-sort passes with device-resident
// element counts, so a pipeline can size its work on the GPU without reading
// counts back to the host.
#pragma once

#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ uint32_t load_n(const uint32_t *n_ptr, uint32_t n_max) {
  if (!n_ptr) return n_max;
  uint32_t n = *n_ptr;
  return n < n_max ? n : n_max;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *excl, uint32_t *smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = THREADS / 32;
    uint32_t w = lane < NW ? smem[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) smem[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t warp_off = wid ? smem[wid - 1] : 0u;
  const uint32_t total = smem[THREADS / 32 - 1];
  *excl = warp_off + x - v;
  __syncthreads();
  return total;
}

// Pass 1: per-tile sums.
template <class Load>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(Load ld, const uint32_t *n_ptr,
                                                                   uint32_t n_max, uint32_t *sums) {
  __shared__ uint32_t smem[32];
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
  uint32_t acc = 0;
  if (base < n) {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const uint32_t i = base + k * kScanThreads + threadIdx.x;  // coalesced
      if (i < n) acc += ld(i);
    }
  }
  uint32_t ex;
  const uint32_t tot = block_exclusive_scan<kScanThreads>(acc, &ex, smem);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Pass 2: exclusive scan of the tile sums in place (one block); total -> *total.
static __global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t *sums, int nblocks, uint32_t *total) {
  __shared__ uint32_t smem[32];
  const int per = (nblocks + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  uint32_t acc = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nblocks) acc += sums[b0 + k];
  uint32_t ex;
  const uint32_t tot = block_exclusive_scan<1024>(acc, &ex, smem);
  for (int k = 0; k < per; ++k) {
    if (b0 + k < nblocks) {
      const uint32_t v = sums[b0 + k];
      sums[b0 + k] = ex;
      ex += v;
    }
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

// Pass 3: per-element exclusive prefix; ap(i, prefix, value) for every i < n and
// ap.end(n, total) once.
template <class Load, class Apply>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(Load ld, Apply ap, const uint32_t *n_ptr,
                                                                  uint32_t n_max, const uint32_t *sums) {
  __shared__ uint32_t smem[32];
  __shared__ uint32_t vals[kScanTile];
  const uint32_t n = load_n(n_ptr, n_max);
  const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
  if (base >= n) {
    if (blockIdx.x == 0) ap.end(n, 0u);
    return;
  }
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t i = base + k * kScanThreads + threadIdx.x;
    vals[k * kScanThreads + threadIdx.x] = i < n ? ld(i) : 0u;
  }
  __syncthreads();
  // each thread owns kScanItems consecutive elements
  uint32_t loc[kScanItems], acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = vals[threadIdx.x * kScanItems + k];
    acc += loc[k];
  }
  uint32_t ex;
  const uint32_t tot = block_exclusive_scan<kScanThreads>(acc, &ex, smem);
  ex += sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t i = base + threadIdx.x * kScanItems + k;
    if (i < n) ap(i, ex, loc[k]);
    ex += loc[k];
  }
  if (base + kScanTile >= n && threadIdx.x == 0) ap.end(n, sums[blockIdx.x] + tot);
}

template <class Load, class Apply>
cudaError_t scan_launch(Load ld, Apply ap, const uint32_t *n_ptr, uint32_t n_max, uint32_t *block_sums,
                        uint32_t *total_out, cudaStream_t s) {
  const int nblocks = (int)((n_max + kScanTile - 1) / kScanTile);
  if (nblocks == 0) {
    // still report an empty result
    scan_apply_kernel<<<1, kScanThreads, 0, s>>>(ld, ap, n_ptr, 0u, block_sums);
    GS_LAUNCHED(1);
    return cudaGetLastError();
  }
  scan_reduce_kernel<<<nblocks, kScanThreads, 0, s>>>(ld, n_ptr, n_max, block_sums);
  scan_sums_kernel<<<1, 1024, 0, s>>>(block_sums, nblocks, total_out);
  scan_apply_kernel<<<nblocks, kScanThreads, 0, s>>>(ld, ap, n_ptr, n_max, block_sums);
  GS_LAUNCHED(3);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort
//
// One LSD pass over (key, value) pairs on 8 bits starting at `shift`. The n
// elements (device count) are split into kSortBlocks contiguous chunks; pass A
// counts digits per chunk, pass B scans the [digit][chunk] table, pass C scatters
// every chunk in order with warp-level stable ranking (match.any), so equal
// digits keep their input order and the sort is stable.

__device__ __forceinline__ void sort_chunk(uint32_t n, uint32_t &lo, uint32_t &hi) {
  const uint32_t tile = kSortThreads * kSortItems;
  uint32_t per = (n + kSortBlocks - 1) / kSortBlocks;
  per = (per + tile - 1) / tile * tile;
  lo = min(n, blockIdx.x * per);
  hi = min(n, lo + per);
}

static __global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t *keys, const uint32_t *n_ptr,
                                                                  uint32_t n_max, int shift,
                                                                  uint32_t *hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  uint32_t lo, hi;
  sort_chunk(load_n(n_ptr, n_max), lo, hi);
  for (uint32_t i = lo + threadIdx.x; i < hi; i += kSortThreads)
    atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[threadIdx.x * kSortBlocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the [digit][block] table in digit-major order. Each warp owns
// 8 digit rows and walks them with coalesced 32-wide loads: row totals first,
// then a scan of the 256 totals, then the in-row prefixes.
static __global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *hist) {
  __shared__ uint32_t row_total[256];
  __shared__ uint32_t smem[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kRowsPerWarp = 256 / 32;
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int d = wid * kRowsPerWarp + r;
    uint32_t acc = 0;
    for (int b = lane; b < kSortBlocks; b += 32) acc += hist[d * kSortBlocks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) row_total[d] = acc;
  }
  __syncthreads();
  uint32_t ex = 0;
  const uint32_t v = threadIdx.x < 256 ? row_total[threadIdx.x] : 0u;
  block_exclusive_scan<1024>(v, &ex, smem);
  if (threadIdx.x < 256) row_total[threadIdx.x] = ex;
  __syncthreads();
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int d = wid * kRowsPerWarp + r;
    uint32_t carry = row_total[d];
    for (int b0 = 0; b0 < kSortBlocks; b0 += 32) {
      const int b = b0 + lane;
      const uint32_t x = b < kSortBlocks ? hist[d * kSortBlocks + b] : 0u;
      uint32_t incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (b < kSortBlocks) hist[d * kSortBlocks + b] = carry + incl - x;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

static __global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint32_t *keys_in,
                                                                     const uint32_t *vals_in,
                                                                     uint32_t *keys_out, uint32_t *vals_out,
                                                                     const uint32_t *n_ptr, uint32_t n_max,
                                                                     int shift, const uint32_t *hist) {
  constexpr int NW = kSortThreads / 32;
  __shared__ uint32_t warp_cnt[NW][256];
  __shared__ uint32_t run[256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t lo, hi;
  sort_chunk(load_n(n_ptr, n_max), lo, hi);
  run[threadIdx.x] = hist[threadIdx.x * kSortBlocks + blockIdx.x];
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (uint32_t t0 = lo; t0 < hi; t0 += kSortThreads * kSortItems) {
    for (int d = threadIdx.x; d < NW * 256; d += kSortThreads) (&warp_cnt[0][0])[d] = 0;
    __syncthreads();
    // each warp owns 32 * kSortItems consecutive items of this tile
    uint32_t k[kSortItems], v[kSortItems], rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t i = t0 + (uint32_t)(wid * 32 * kSortItems + r * 32 + lane);
      const bool ok = i < hi;
      k[r] = ok ? keys_in[i] : 0u;
      v[r] = ok ? vals_in[i] : 0u;
      const uint32_t dig = ok ? (k[r] >> shift) & 255u : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, dig);
      const uint32_t before = ok ? warp_cnt[wid][dig] : 0u;
      rank[r] = before + __popc(peers & lt_mask);
      __syncwarp();
      if (ok && (peers & lt_mask) == 0) warp_cnt[wid][dig] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {  // per digit: offsets of each warp's items, then advance the running offset
      const int d = threadIdx.x;
      uint32_t acc = run[d];
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = warp_cnt[w][d];
        warp_cnt[w][d] = acc;
        acc += c;
      }
      run[d] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t i = t0 + (uint32_t)(wid * 32 * kSortItems + r * 32 + lane);
      if (i < hi) {
        const uint32_t dig = (k[r] >> shift) & 255u;
        const uint32_t pos = warp_cnt[wid][dig] + rank[r];
        keys_out[pos] = k[r];
        vals_out[pos] = v[r];
      }
    }
    __syncthreads();
  }
}

// Sorts (keys, vals) on bits [0, bits) with ceil(bits/8) passes; the result
// lands in buffer index `*which` (0 or 1) of the double buffers.
inline cudaError_t radix_sort(uint32_t *const keys[2], uint32_t *const vals[2], const uint32_t *n_ptr, uint32_t n_max,
                              int bits, uint32_t *hist, int *which, cudaStream_t s) {
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<kSortBlocks, kSortThreads, 0, s>>>(keys[cur], n_ptr, n_max, shift, hist);
    radix_scan_kernel<<<1, 1024, 0, s>>>(hist);
    radix_scatter_kernel<<<kSortBlocks, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                               vals[cur ^ 1], n_ptr, n_max, shift, hist);
    GS_LAUNCHED(3);
    cur ^= 1;
  }
  *which = cur;
  return cudaGetLastError();
}

}  // namespace gs
