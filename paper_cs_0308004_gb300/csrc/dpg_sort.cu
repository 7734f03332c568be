// The three-phase main-memory sort of §3 on sm_103a: (1) extract key-pointer
// pairs, (2) sort the pairs, (3) copy the records into key order.  Phase 3 is
// record retrieval (dpg_retrieve.cu); this file holds phases 1 and 2.
//
// Pair layout (16 bytes): bytes [0, key_bytes) the record's key, zero padding
// up to byte 12, the int32 rid at byte 12.  Keys compare as unsigned byte
// strings; equal keys keep rid order.
//
// Phase 2 is a stable least-significant-digit radix sort with one key byte
// per pass (byte key_bytes-1 first, byte 0 last).  Every key byte's digits
// are counted over all pairs once, by the kernel that builds the pairs
// (k_extract_pairs here, the join's k_extract_fk_pairs): the counts do not
// depend on the order.  Each pass is then one kernel, k_rs_onesweep: a CTA
// takes the next tile (64 KB of pairs), ranks its pairs stably (per-warp
// digit counts, the lanes sharing a digit found with a shared-memory OR, a
// prefix over warps), publishes the tile's digit counts, finds how many pairs
// of each digit earlier tiles hold by looking back over their published
// counts (decoupled look-back; every wait is bounded), then reorders the tile
// in shared memory and writes each digit's pairs as one contiguous piece at
// digit base + earlier tiles' count.
#include <algorithm>

#include "dpg_device.cuh"
#include "dpg_internal.h"

namespace dpg {
namespace {

// Tiles of 4096 16-byte or 8192 8-byte pairs (64 KB), two CTAs per SM: the
// fewer tiles per byte, the fewer look-back walks and block barriers (4096
// 16-byte pairs: 109 against 138 us per pass over 1e7 pairs for 2048 at three
// CTAs per SM).
constexpr int kRsThreads = 512;
constexpr int kRsMinBlocks = 2;
constexpr int kRsWarps = kRsThreads / 32;
template <class E> __host__ __device__ constexpr int rs_items() { return sizeof(E) == 16 ? 8 : 16; }
// pairs per tile
template <class E> __host__ __device__ constexpr uint32_t rs_tile() { return kRsThreads * rs_items<E>(); }

// Phase 1: pairs[i] = (key of record i, zero pad, i).  WORDS: records and
// the table are 4-byte aligned, so the key is read as ceil(key_bytes/4)
// words (never past the record: key_bytes <= rec, rec a multiple of 4).
// The digit counts of every key byte (counts[j * 256 + d], zero on entry)
// are taken on the way, so the radix sort need not read the pairs for them.
template <bool WORDS>
__global__ void __launch_bounds__(256)
    k_extract_pairs(const uint8_t* __restrict__ src, uint64_t n, uint32_t rec, uint32_t key_bytes,
                    uint4* __restrict__ pairs, uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[12 * 256];
  for (uint32_t x = threadIdx.x; x < key_bytes * 256; x += blockDim.x) h[x] = 0;
  __syncthreads();
  const uint32_t nw = (key_bytes + 3) / 4;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t* r = src + i * rec;
    uint32_t w[4] = {0u, 0u, 0u, (uint32_t)i};
    if (WORDS) {
      const uint32_t* rw = reinterpret_cast<const uint32_t*>(r);
#pragma unroll
      for (uint32_t j = 0; j < 3; ++j)
        if (j < nw) {
          const uint32_t keep = key_bytes >= 4 * (j + 1) ? 32u : 8u * (key_bytes - 4 * j);
          const uint32_t v = __ldg(rw + j);
          w[j] = keep == 32u ? v : (v & ((1u << keep) - 1u));
        }
    } else {
#pragma unroll
      for (uint32_t b = 0; b < 12; ++b)
        if (b < key_bytes) w[b >> 2] |= (uint32_t)__ldg(r + b) << (8 * (b & 3));
    }
    pairs[i] = make_uint4(w[0], w[1], w[2], w[3]);
    for (uint32_t j = 0; j < key_bytes; ++j) atomicAdd(&h[j * 256 + ((w[j >> 2] >> (8 * (j & 3))) & 0xffu)], 1u);
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < key_bytes * 256; x += blockDim.x)
    if (h[x]) atomicAdd(&counts[x], h[x]);
}

// Key byte `byte` of a pair: 16-byte pairs hold up to 12 key bytes in words
// x, y, z; 8-byte pairs (the DPG-sort join's) up to 4 in x, the rid in y.
__device__ __forceinline__ uint32_t pair_digit(const uint4& p, uint32_t byte) {
  const uint32_t word = byte < 4 ? p.x : (byte < 8 ? p.y : p.z);
  return (word >> (8 * (byte & 3))) & 0xffu;
}
__device__ __forceinline__ uint32_t pair_digit(const uint2& p, uint32_t byte) {
  return (p.x >> (8 * (byte & 3))) & 0xffu;
}

constexpr uint32_t kFlagAgg = 1u << 30, kFlagPrefix = 2u << 30, kCountMask = (1u << 30) - 1;

// One stable pass on key byte `byte`.  Tiles are numbered in the order CTAs
// start (tile_ctr), so a tile only waits for tiles whose CTAs already run.
// E: uint4 (16-byte pairs) or uint2 (8-byte pairs).
template <class E>
__global__ void __launch_bounds__(kRsThreads, kRsMinBlocks)
    k_rs_onesweep(const E* __restrict__ in, E* __restrict__ out, uint64_t n, uint32_t byte,
                  const uint32_t* __restrict__ digit_count, uint32_t* status, uint32_t* tile_ctr, int* err,
                  long long wait_limit) {
  __shared__ uint16_t whist[kRsWarps][256];
  __shared__ uint32_t wmask[kRsWarps][256];  // lanes of a warp holding digit d in this round
  __shared__ uint32_t tcnt[256], toff[256], s_base[256], s_excl[256];
  __shared__ uint32_t s_tile;
  constexpr int kItems = rs_items<E>();
  constexpr uint32_t kTile = rs_tile<E>();
  extern __shared__ uint4 sraw[];
  E* sbuf = reinterpret_cast<E*>(sraw);                      // kTile pairs
  uint8_t* sdig = reinterpret_cast<uint8_t*>(sbuf + kTile);  // kTile digits
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (uint32_t x = threadIdx.x; x < kRsWarps * 256; x += kRsThreads) {
    (&whist[0][0])[x] = 0;
    (&wmask[0][0])[x] = 0;
  }
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kTile;
  // digit bases of this pass: exclusive scan of the digit counts (warp 1, 8 per lane)
  if (warp == 1) {
    uint32_t c[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = digit_count[lane * 8 + j];
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
      s_base[lane * 8 + j] = run;
      run += c[j];
    }
  }
  // this thread's pairs: kItems rounds of 32 consecutive pairs of its warp
  // (the digit is recomputed from the pair where it is needed)
  const uint64_t e0 = base + (uint64_t)warp * (32 * kItems) + lane;
  E v[kItems];
  uint32_t rank[kItems];
  // all of the tile's loads first: the ranking below has warp barriers,
  // which would otherwise hold each load back until the previous round ends
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if (e0 + (uint64_t)k * 32 < n) v[k] = in[e0 + (uint64_t)k * 32];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const bool ok = e0 + (uint64_t)k * 32 < n;
    const uint32_t d = ok ? pair_digit(v[k], byte) : 0u;
    // peers: the lanes of this warp with the same digit, gathered by a
    // shared-memory OR (cheaper here than __match_any_sync)
    if (ok) atomicOr(&wmask[warp][d], 1u << lane);
    __syncwarp();
    const uint32_t peers = ok ? wmask[warp][d] : (1u << lane);
    const uint32_t before = __popc(peers & lt);
    uint32_t prior = 0;
    if (ok) prior = whist[warp][d];
    __syncwarp();
    if (ok && before == 0) {
      whist[warp][d] = (uint16_t)(prior + __popc(peers));
      wmask[warp][d] = 0;
    }
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
    // publish this tile's count of digit d, then look back over earlier tiles
    volatile uint32_t* st = status;
    const uint32_t dg = threadIdx.x;
    st[(uint64_t)t * 256 + dg] = (t == 0 ? kFlagPrefix : kFlagAgg) | run;
    uint32_t excl = 0;
    if (t > 0) {
      // tile j < t was claimed before this one, so its CTA is running and
      // publishes its count; the wait is bounded all the same
      for (int64_t j = (int64_t)t - 1; j >= 0; --j) {
        bool ok;
        const uint32_t w = wait_word_bounded(status + (uint64_t)j * 256 + dg, wait_limit, &ok,
                                             [](uint32_t x) { return (x & ~kCountMask) != 0; });
        if (!ok) {
          atomicOr(err, ERR_TIMEOUT);
          break;
        }
        excl += w & kCountMask;
        if ((w & ~kCountMask) == kFlagPrefix) break;
      }
      st[(uint64_t)t * 256 + dg] = kFlagPrefix | (excl + run);
    }
    s_excl[dg] = excl;
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the tile's 256 digit counts, 8 per lane
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
  for (int k = 0; k < kItems; ++k) {
    if (e0 + (uint64_t)k * 32 < n) {
      const uint32_t d = pair_digit(v[k], byte);
      const uint32_t p = toff[d] + whist[warp][d] + rank[k];
      sbuf[p] = v[k];
      sdig[p] = (uint8_t)d;
    }
  }
  __syncthreads();
  const uint32_t tn = (uint32_t)((n - base) < kTile ? (n - base) : kTile);
  for (uint32_t p = threadIdx.x; p < tn; p += kRsThreads) {
    const uint32_t dg = sdig[p];
    out[(uint64_t)s_base[dg] + s_excl[dg] + (p - toff[dg])] = sbuf[p];
  }
}

}  // namespace

// Phases 1 and 2 of §3: sorted key-pointer pairs of src into `pairs`
// (n_src x 16 bytes).  `tmp` is n_src x 16 bytes of scratch; `scan` holds the
// digit-count matrix (12 x 256 words at its start), the tile counter and the
// tiles' published counts (see sort_scan_bytes).
size_t sort_scan_bytes(uint64_t n) {
  const uint64_t ntiles = (n + rs_tile<uint4>() - 1) / rs_tile<uint4>();  // the smaller tile: the most tiles
  return ((256 * ntiles * 4 + 255) & ~255ull) + 16384;
}

namespace {

template <class E>
uint8_t* radix_pairs(dpg_ctx& ctx, uint8_t* a_, uint8_t* b_, uint8_t* scan, uint64_t n, uint32_t key_bytes,
                     cudaStream_t st, int* status) {
  *status = DPG_OK;
  E* a = reinterpret_cast<E*>(a_);
  E* b = reinterpret_cast<E*>(b_);
  if (n == 0) return a_;
  if (n > kCountMask || key_bytes > (sizeof(E) == 16 ? 12u : 4u)) {
    *status = DPG_EINVAL;
    return nullptr;
  }
  const uint32_t ntiles = (uint32_t)((n + rs_tile<E>() - 1) / rs_tile<E>());
  const uint32_t* counts = radix_counts(scan);  // key_bytes x 256, filled by the caller
  uint32_t* tile_ctr = radix_counts(scan) + 12 * 256;
  uint32_t* tile_status = reinterpret_cast<uint32_t*>(scan + 16384);
  cudaError_t e = cudaSuccess;
  const size_t smem = rs_tile<E>() * (sizeof(E) + 1);
  cudaFuncSetAttribute(k_rs_onesweep<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int byte = (int)key_bytes - 1; byte >= 0; --byte) {
    e = cudaMemsetAsync(tile_status, 0, (size_t)ntiles * 256 * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tile_ctr, 0, 4, st);
    if (e != cudaSuccess) {
      *status = cuda_fail(ctx, e, "memset");
      return nullptr;
    }
    {
      TraceScope ts(ctx, "k_rs_onesweep", st);
      k_rs_onesweep<E><<<ntiles, kRsThreads, smem, st>>>(a, b, n, (uint32_t)byte, counts + 256 * byte, tile_status,
                                                        tile_ctr, ctx.d_err, ctx.wait_cycles);
    }
    ctx.launches++;
    std::swap(a, b);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) *status = cuda_fail(ctx, e, "sort launch");
  return reinterpret_cast<uint8_t*>(a);
}

}  // namespace

uint32_t* radix_counts(uint8_t* scan) { return reinterpret_cast<uint32_t*>(scan); }

uint8_t* run_radix_pairs(dpg_ctx& ctx, uint8_t* a, uint8_t* b, uint8_t* scan, uint64_t n, uint32_t key_bytes,
                         cudaStream_t st, int* status) {
  return radix_pairs<uint4>(ctx, a, b, scan, n, key_bytes, st, status);
}

uint8_t* run_radix_pairs8(dpg_ctx& ctx, uint8_t* a, uint8_t* b, uint8_t* scan, uint64_t n, uint32_t key_bytes,
                          cudaStream_t st, int* status) {
  return radix_pairs<uint2>(ctx, a, b, scan, n, key_bytes, st, status);
}

int run_sort_keyptr(dpg_ctx& ctx, const uint8_t* src, uint64_t n, uint32_t rec, uint32_t key_bytes, uint8_t* pairs,
                    uint8_t* tmp, uint8_t* scan, cudaStream_t st) {
  if (n == 0) return DPG_OK;
  // an even number of passes ends where it started
  uint8_t* start = (key_bytes % 2 == 0) ? pairs : tmp;
  uint8_t* other = (key_bytes % 2 == 0) ? tmp : pairs;
  if (key_bytes == 0 || key_bytes > 12) return DPG_EINVAL;
  uint32_t* counts = radix_counts(scan);
  cudaError_t e = cudaMemsetAsync(counts, 0, 12 * 256 * 4, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  {
    TraceScope ts(ctx, "k_extract_pairs", st);
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx.sms * 8);
    if (rec % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 4 == 0)
      k_extract_pairs<true><<<grid, 256, 0, st>>>(src, n, rec, key_bytes, reinterpret_cast<uint4*>(start), counts);
    else
      k_extract_pairs<false><<<grid, 256, 0, st>>>(src, n, rec, key_bytes, reinterpret_cast<uint4*>(start), counts);
    ctx.launches++;
  }
  int status = DPG_OK;
  run_radix_pairs(ctx, start, other, scan, n, key_bytes, st, &status);
  return status;
}

}  // namespace dpg
