// Scan kernels shared by the retrieval (Phase I) and the radix sort: turn a
// bucket-major count matrix cnt[b*G + g] (b: bucket / run / digit, g: CTA or
// tile) into write cursors off[b] + sum_{g' < g} cnt[b*G + g'], plus bucket
// offsets and probe work-item offsets.
#pragma once

#include <cstdint>

#include "dpg_device.cuh"

namespace dpg {
namespace {

constexpr uint32_t kScanTile = 1024;  // segments per tile of the two-level scan

// K3a: block x owns segments [32x, 32x+32), one warp per segment.  In
// shared-counter mode each warp sums its row of the count matrix into tot[b];
// the block then adds its segments' rid counts and probe work items
// (ceil(count / chunk)) to the sums of their tile of kScanTile segments
// (tsum, isum: zeroed before the launch).
__global__ void __launch_bounds__(1024)
    k_bucket_totals(const uint32_t* __restrict__ cnt, uint32_t* __restrict__ tot, uint32_t nb, uint32_t G,
                    uint32_t chunk, uint32_t* __restrict__ tsum, uint32_t* __restrict__ isum, const int* err,
                    int smem_mode) {
  __shared__ uint32_t s_t[32], s_i[32];
  if (error_set(err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t b = blockIdx.x * 32 + warp;
  uint32_t t = 0;
  if (b < nb) {
    if (smem_mode) {
      const uint32_t* row = cnt + (uint64_t)b * G;
      for (uint32_t c = lane; c < G; c += 32) t += row[c];
#pragma unroll
      for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) tot[b] = t;
    } else {
      t = tot[b];
    }
  }
  if (lane == 0) {
    s_t[warp] = t;
    s_i[warp] = (t + chunk - 1) / chunk;
  }
  __syncthreads();
  if (warp == 0) {
    uint32_t x = s_t[lane], y = s_i[lane];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      const uint32_t tile = blockIdx.x * 32 / kScanTile;
      atomicAdd(&tsum[tile], x);
      atomicAdd(&isum[tile], y);
    }
  }
}

// K3b: block x owns segments [32x, 32x+32).  It adds the tile sums of earlier
// tiles and the counts of earlier segments of its own tile, scans its 32
// segments (off[], itemoff[]), then each warp turns one row of the count
// matrix into write cursors: cnt[b*G + g] <- off[b] + sum_{g' < g} cnt[b*G + g'].
__global__ void __launch_bounds__(1024)
    k_scan(const uint32_t* __restrict__ tot, const uint32_t* __restrict__ tsum, const uint32_t* __restrict__ isum,
           uint32_t nb, uint32_t G, uint32_t chunk, uint32_t* __restrict__ cnt, uint32_t* __restrict__ off,
           uint32_t* __restrict__ itemoff, uint32_t* item_counter, const int* err) {
  __shared__ uint32_t s_t[32], s_i[32], s_off[32];
  if (error_set(err)) return;
  const uint32_t b0 = blockIdx.x * 32;
  const uint32_t tile = b0 / kScanTile, tile_start = tile * kScanTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t st = 0, si = 0;
  for (uint32_t x = threadIdx.x; x < tile; x += blockDim.x) {
    st += tsum[x];
    si += isum[x];
  }
  for (uint32_t b = tile_start + threadIdx.x; b < b0; b += blockDim.x) {
    const uint32_t t = tot[b];
    st += t;
    si += (t + chunk - 1) / chunk;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    st += __shfl_xor_sync(0xffffffffu, st, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    s_t[warp] = st;
    s_i[warp] = si;
  }
  __syncthreads();
  if (warp == 0) {
    uint32_t a = s_t[lane], c = s_i[lane];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const uint32_t b = b0 + lane;
    const uint32_t t = b < nb ? tot[b] : 0;
    const uint32_t it = (t + chunk - 1) / chunk;
    uint32_t ti = t, ii = it;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, ti, o), y = __shfl_up_sync(0xffffffffu, ii, o);
      if (lane >= o) {
        ti += x;
        ii += y;
      }
    }
    const uint32_t eo = a + ti - t, ei = c + ii - it;
    s_off[lane] = eo;
    if (b < nb) {
      off[b] = eo;
      itemoff[b] = ei;
    }
    if (b + 1 == nb) {
      off[nb] = a + ti;
      itemoff[nb] = c + ii;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *item_counter = 0;
  __syncthreads();
  const uint32_t b = b0 + warp;
  if (b < nb) {
    uint32_t run = s_off[warp];
    uint32_t* row = cnt + (uint64_t)b * G;
    for (uint32_t c0 = 0; c0 < G; c0 += 32) {
      const uint32_t c = c0 + lane;
      const uint32_t v = c < G ? row[c] : 0;
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      if (c < G) row[c] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

}  // namespace
}  // namespace dpg
