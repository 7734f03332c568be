// The three-phase main-memory sort of §3 on sm_103a: (1) extract key-pointer
// pairs, (2) sort the pairs, (3) copy the records into key order.  Phase 3 is
// record retrieval (dpg_retrieve.cu); this file holds phases 1 and 2.
//
// Pair layout (16 bytes): bytes [0, key_bytes) the record's key, zero padding
// up to byte 12, the int32 rid at byte 12.  Keys compare as unsigned byte
// strings; equal keys keep rid order.
//
// Phase 2 is a stable least-significant-digit radix sort with one key byte
// per pass (byte key_bytes-1 first, byte 0 last).  Each pass: k_rs_hist counts
// the digit of every pair per tile of kRsTile pairs (digit-major count matrix),
// the shared scan kernels turn the counts into per-(digit, tile) cursors, and
// k_rs_scatter ranks the tile's pairs stably (per-warp digit counts built with
// __match_any_sync, prefix over warps), reorders the tile in shared memory and
// writes each digit's pairs as one contiguous piece.
#include <algorithm>

#include "dpg_device.cuh"
#include "dpg_internal.h"
#include "dpg_scan.cuh"

namespace dpg {
namespace {

constexpr int kRsThreads = 1024;
constexpr int kRsItems = 4;
constexpr uint32_t kRsTile = kRsThreads * kRsItems;  // pairs per tile
constexpr int kRsWarps = kRsThreads / 32;

// Phase 1: pairs[i] = (key of record i, zero pad, i).
__global__ void __launch_bounds__(256)
    k_extract_pairs(const uint8_t* __restrict__ src, uint64_t n, uint32_t rec, uint32_t key_bytes,
                    uint4* __restrict__ pairs) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t* r = src + i * rec;
    uint32_t w[4] = {0u, 0u, 0u, (uint32_t)i};
#pragma unroll
    for (uint32_t b = 0; b < 12; ++b)
      if (b < key_bytes) w[b >> 2] |= (uint32_t)__ldg(r + b) << (8 * (b & 3));
    pairs[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__device__ __forceinline__ uint32_t pair_digit(const uint4& p, uint32_t byte) {
  const uint32_t word = byte < 4 ? p.x : (byte < 8 ? p.y : p.z);
  return (word >> (8 * (byte & 3))) & 0xffu;
}

// Per-tile digit counts: cnt[d * ntiles + tile].
__global__ void __launch_bounds__(kRsThreads)
    k_rs_hist(const uint4* __restrict__ in, uint64_t n, uint32_t byte, uint32_t ntiles, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t h[256];
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (threadIdx.x < 256) h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)t * kRsTile;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const uint64_t e = base + (uint64_t)k * kRsThreads + threadIdx.x;
      if (e < n) atomicAdd(&h[pair_digit(in[e], byte)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 256) cnt[(uint64_t)threadIdx.x * ntiles + t] = h[threadIdx.x];
    __syncthreads();
  }
}

// Stable scatter of one tile by digit.  Warp w owns tile elements
// [128w, 128w + 128) taken in order (k major, lane minor), so the rank of an
// element among equal digits is: its rank inside its warp step, plus the
// equal digits of earlier steps of its warp, plus those of earlier warps.
__global__ void __launch_bounds__(kRsThreads)
    k_rs_scatter(const uint4* __restrict__ in, uint4* __restrict__ out, uint64_t n, uint32_t byte, uint32_t ntiles,
                 const uint32_t* __restrict__ cur) {
  __shared__ uint16_t whist[kRsWarps][256];
  __shared__ uint32_t tcnt[256], toff[256];
  extern __shared__ uint4 sbuf[];                              // kRsTile pairs
  uint8_t* sdig = reinterpret_cast<uint8_t*>(sbuf + kRsTile);  // kRsTile digits
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (uint32_t x = threadIdx.x; x < kRsWarps * 256; x += kRsThreads) (&whist[0][0])[x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)t * kRsTile;
    uint4 v[kRsItems];
    uint32_t d[kRsItems], rank[kRsItems];
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const uint64_t e = base + (uint64_t)warp * (32 * kRsItems) + (uint64_t)k * 32 + lane;
      const bool ok = e < n;
      if (ok) v[k] = in[e];
      d[k] = ok ? pair_digit(v[k], byte) : 256u + lane;  // unique sentinel per lane past the end
      const uint32_t peers = __match_any_sync(0xffffffffu, d[k]);
      const uint32_t before = __popc(peers & lt);
      uint32_t prior = 0;
      if (ok) prior = whist[warp][d[k]];
      __syncwarp();
      if (ok && before == 0) whist[warp][d[k]] = (uint16_t)(prior + __popc(peers));
      __syncwarp();
      rank[k] = prior + before;
    }
    __syncthreads();
    if (threadIdx.x < 256) {  // exclusive prefix over warps, per digit
      uint32_t run = 0;
      for (int w = 0; w < kRsWarps; ++w) {
        const uint32_t c = whist[w][threadIdx.x];
        whist[w][threadIdx.x] = (uint16_t)run;
        run += c;
      }
      tcnt[threadIdx.x] = run;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 256 digit counts, 8 per lane
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        c[j] = tcnt[lane * 8 + j];
        sum += c[j];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - sum;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        toff[lane * 8 + j] = run;
        run += c[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      if (d[k] < 256u) {
        const uint32_t p = toff[d[k]] + whist[warp][d[k]] + rank[k];
        sbuf[p] = v[k];
        sdig[p] = (uint8_t)d[k];
      }
    }
    __syncthreads();
    const uint32_t tn = (uint32_t)((n - base) < kRsTile ? (n - base) : kRsTile);
    for (uint32_t p = threadIdx.x; p < tn; p += kRsThreads) {
      const uint32_t dg = sdig[p];
      out[cur[(uint64_t)dg * ntiles + t] + (p - toff[dg])] = sbuf[p];
    }
    __syncthreads();
  }
}

}  // namespace

// Phases 1 and 2 of §3: sorted key-pointer pairs of src into `pairs`
// (n_src x 16 bytes).  `tmp` is n_src x 16 bytes of scratch; `scan` holds the
// count matrix and scan buffers (see sort_scan_bytes).
size_t sort_scan_bytes(uint64_t n) {
  const uint64_t ntiles = (n + kRsTile - 1) / kRsTile;
  return ((256 * ntiles * 4 + 255) & ~255ull) + 4096;
}

uint8_t* run_radix_pairs(dpg_ctx& ctx, uint8_t* a_, uint8_t* b_, uint8_t* scan, uint64_t n, uint32_t key_bytes,
                         cudaStream_t st, int* status) {
  *status = DPG_OK;
  uint4* a = reinterpret_cast<uint4*>(a_);
  uint4* b = reinterpret_cast<uint4*>(b_);
  if (n == 0) return a_;
  const uint32_t ntiles = (uint32_t)((n + kRsTile - 1) / kRsTile);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(scan);
  uint8_t* rest = scan + ((256ull * ntiles * 4 + 255) & ~255ull);
  uint32_t* tot = reinterpret_cast<uint32_t*>(rest);  // 256
  uint32_t* off = tot + 256;                            // 257
  uint32_t* itemoff = off + 260;                        // 257
  uint32_t* tsum = itemoff + 260;                       // 1 (+pad)
  uint32_t* isum = tsum + 4;                            // 1 (+pad)
  uint32_t* counter = isum + 4;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx.sms * 2);
  const size_t smem = kRsTile * (sizeof(uint4) + 1);
  cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int byte = (int)key_bytes - 1; byte >= 0; --byte) {
    {
      TraceScope ts(ctx, "k_rs_hist", st);
      k_rs_hist<<<grid, kRsThreads, 0, st>>>(a, n, (uint32_t)byte, ntiles, cnt);
    }
    cudaError_t e = cudaMemsetAsync(tsum, 0, 32, st);
    if (e != cudaSuccess) {
      *status = cuda_fail(ctx, e, "memset");
      return nullptr;
    }
    {
      TraceScope ts(ctx, "k_rs_scan", st);
      k_bucket_totals<<<256 / 32, 1024, 0, st>>>(cnt, tot, 256, ntiles, 1u << 30, tsum, isum, ctx.d_err, 1);
      k_scan<<<256 / 32, 1024, 0, st>>>(tot, tsum, isum, 256, ntiles, 1u << 30, cnt, off, itemoff, counter,
                                        ctx.d_err);
    }
    {
      TraceScope ts(ctx, "k_rs_scatter", st);
      k_rs_scatter<<<grid, kRsThreads, smem, st>>>(a, b, n, (uint32_t)byte, ntiles, cnt);
    }
    ctx.launches += 4;
    std::swap(a, b);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) *status = cuda_fail(ctx, e, "sort launch");
  return reinterpret_cast<uint8_t*>(a);
}

int run_sort_keyptr(dpg_ctx& ctx, const uint8_t* src, uint64_t n, uint32_t rec, uint32_t key_bytes, uint8_t* pairs,
                    uint8_t* tmp, uint8_t* scan, cudaStream_t st) {
  if (n == 0) return DPG_OK;
  // an even number of passes ends where it started
  uint8_t* start = (key_bytes % 2 == 0) ? pairs : tmp;
  uint8_t* other = (key_bytes % 2 == 0) ? tmp : pairs;
  {
    TraceScope ts(ctx, "k_extract_pairs", st);
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx.sms * 8);
    k_extract_pairs<<<grid, 256, 0, st>>>(src, n, rec, key_bytes, reinterpret_cast<uint4*>(start));
    ctx.launches++;
  }
  int status = DPG_OK;
  run_radix_pairs(ctx, start, other, scan, n, key_bytes, st, &status);
  return status;
}

}  // namespace dpg
