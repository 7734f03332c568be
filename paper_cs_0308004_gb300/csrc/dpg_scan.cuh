// Phase I scan kernels of the retrieval: turn the CTA-major count matrix
// cnt[g*nb + b] (g: Phase I CTA, b: segment) into write cursors
// off[b] + sum_{g' < g} cnt[g'*nb + b], plus the segment offsets off[] and
// the probe work-item offsets itemoff[].
//
// CTA-major rows let every Phase I CTA write (and later read back) its nb
// counters as one contiguous row.  Both kernels here read the matrix with
// lanes on consecutive segments: a block owns kScanBlock segments, split into
// groups of 32 (one lane per segment), and the CTAs g into kScanSlices
// slices, one warp per (group, slice).
#pragma once

#include <cstdint>

#include "dpg_device.cuh"

namespace dpg {
namespace {

constexpr uint32_t kScanTile = 1024;   // segments per tile of the two-level scan
constexpr uint32_t kScanBlock = 128;   // segments per block of K3a / K3b
constexpr uint32_t kScanGroups = kScanBlock / 32;
constexpr uint32_t kScanSlices = 1024 / 32 / kScanGroups;  // warps per group
static_assert(kScanTile % kScanBlock == 0, "a block lies inside one tile");

__device__ __forceinline__ void scan_slice(uint32_t G, uint32_t s, uint32_t& g0, uint32_t& g1) {
  const uint32_t per = (G + kScanSlices - 1) / kScanSlices;
  g0 = min(G, s * per);
  g1 = min(G, g0 + per);
}

// K3a: segment totals.  In shared-counter mode (G CTAs) warp (q, s) sums the
// counts of its 32 segments over its slice of CTAs, stores the slice sums in
// psum[s*nb + b] for K3b, and the block combines them into tot[b]; otherwise
// (G == 1, global counters) tot[] is already complete.  The block then adds
// its segments' rid counts and probe work items (ceil(count / chunk)) to the
// sums of its tile of kScanTile segments (tsum, isum: zeroed before launch).
__global__ void __launch_bounds__(1024)
    k_bucket_totals(const uint32_t* __restrict__ cnt, uint32_t* __restrict__ tot, uint32_t* __restrict__ psum,
                    uint32_t nb, uint32_t G, uint32_t chunk, uint32_t* __restrict__ tsum,
                    uint32_t* __restrict__ isum, const int* err, int smem_mode) {
  __shared__ uint32_t part[kScanSlices][kScanBlock];
  if (error_set(err)) return;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t q = warp % kScanGroups, s = warp / kScanGroups;
  const uint32_t b0 = blockIdx.x * kScanBlock;
  const uint32_t b = b0 + q * 32 + lane;
  if (smem_mode) {
    uint32_t t = 0;
    if (b < nb) {
      uint32_t g0, g1;
      scan_slice(G, s, g0, g1);
      uint32_t g = g0;
      for (; g + 4 <= g1; g += 4) {
        const uint32_t* p = cnt + (uint64_t)g * nb + b;
        t += p[0] + p[nb] + p[2 * (uint64_t)nb] + p[3 * (uint64_t)nb];
      }
      for (; g < g1; ++g) t += cnt[(uint64_t)g * nb + b];
      psum[(uint64_t)s * nb + b] = t;
    }
    part[s][q * 32 + lane] = t;
  }
  __syncthreads();
  if (warp >= kScanGroups) return;  // warps 0..3: q == warp, s == 0
  uint32_t t = 0;
  if (b < nb) {
    if (smem_mode) {
#pragma unroll
      for (uint32_t k = 0; k < kScanSlices; ++k) t += part[k][q * 32 + lane];
      tot[b] = t;
    } else {
      t = tot[b];
    }
  }
  uint32_t x = t, y = (t + chunk - 1) / chunk;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  if (lane == 0) {
    const uint32_t tile = b0 / kScanTile;
    atomicAdd(&tsum[tile], x);
    atomicAdd(&isum[tile], y);
  }
}

// K3b: block x owns segments [b0, b0 + kScanBlock), b0 = kScanBlock * x.  It
// adds the tile sums of earlier tiles and the totals of earlier segments of
// its own tile, scans its segments into off[] and itemoff[], then warp (q, s)
// turns its slice of the count columns into write cursors, starting from
// off[b] plus the slice sums psum[] of earlier slices.
__global__ void __launch_bounds__(1024)
    k_scan(const uint32_t* __restrict__ tot, const uint32_t* __restrict__ psum, const uint32_t* __restrict__ tsum,
           const uint32_t* __restrict__ isum, uint32_t nb, uint32_t G, uint32_t chunk, uint32_t* __restrict__ cnt,
           uint32_t* __restrict__ off, uint32_t* __restrict__ itemoff, uint32_t* item_counter, const int* err,
           int smem_mode) {
  __shared__ uint32_t s_t[32], s_i[32], s_off[kScanBlock], s_wt[kScanGroups], s_wi[kScanGroups];
  if (error_set(err)) return;
  const uint32_t b0 = blockIdx.x * kScanBlock;
  const uint32_t tile = b0 / kScanTile, tile_start = tile * kScanTile;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  // inclusive scans of the block's segment totals, one warp per group of 32
  uint32_t t = 0, it = 0, ti = 0, ii = 0;
  if (warp < kScanGroups) {
    const uint32_t b = b0 + warp * 32 + lane;
    t = b < nb ? tot[b] : 0;
    it = (t + chunk - 1) / chunk;
    ti = t;
    ii = it;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, ti, o), y = __shfl_up_sync(0xffffffffu, ii, o);
      if (lane >= o) {
        ti += x;
        ii += y;
      }
    }
    if (lane == 31) {
      s_wt[warp] = ti;
      s_wi[warp] = ii;
    }
  }
  __syncthreads();
  if (warp < kScanGroups) {
    uint32_t a = 0, c = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      a += s_t[k];
      c += s_i[k];
    }
    for (uint32_t k = 0; k < warp; ++k) {
      a += s_wt[k];
      c += s_wi[k];
    }
    const uint32_t b = b0 + warp * 32 + lane;
    const uint32_t eo = a + ti - t, ei = c + ii - it;
    s_off[warp * 32 + lane] = eo;
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
  const uint32_t q = warp % kScanGroups, s = warp / kScanGroups;
  const uint32_t b = b0 + q * 32 + lane;
  if (b >= nb) return;
  if (!smem_mode) {  // G == 1: the cursor is the segment offset
    if (s == 0) cnt[b] = s_off[q * 32 + lane];
    return;
  }
  uint32_t run = s_off[q * 32 + lane];
  for (uint32_t k = 0; k < s; ++k) run += psum[(uint64_t)k * nb + b];
  uint32_t g0, g1;
  scan_slice(G, s, g0, g1);
  uint32_t g = g0;
  for (; g + 4 <= g1; g += 4) {
    uint32_t* p = cnt + (uint64_t)g * nb + b;
    const uint32_t v0 = p[0], v1 = p[nb], v2 = p[2 * (uint64_t)nb], v3 = p[3 * (uint64_t)nb];
    p[0] = run;
    p[nb] = run + v0;
    p[2 * (uint64_t)nb] = run + v0 + v1;
    p[3 * (uint64_t)nb] = run + v0 + v1 + v2;
    run += v0 + v1 + v2 + v3;
  }
  for (; g < g1; ++g) {
    const uint32_t v = cnt[(uint64_t)g * nb + b];
    cnt[(uint64_t)g * nb + b] = run;
    run += v;
  }
}

}  // namespace
}  // namespace dpg
