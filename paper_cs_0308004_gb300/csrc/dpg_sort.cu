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
// digit counts; the lanes sharing a digit are the AND of eight ballots, one
// per digit bit), publishes the tile's digit counts, finds how many pairs of
// each digit earlier tiles hold by looking back over their published counts
// (decoupled look-back; every wait is bounded) while the other half of the
// CTA lays the tile out, then reorders the tile in shared memory and writes
// each digit's pairs as one contiguous piece at digit base + earlier tiles'
// count.
//
// Keys longer than two bytes take only the passes on bytes 1 and 0; each
// bucket of equal two-byte prefix is then sorted on its own (run_sort_keyptr).
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
// earlier tiles read per step of the look-back: 8 for 16-byte pairs (3 us
// less per pass over 1e7 pairs than 1); 1 for 8-byte pairs, whose 16 pairs
// per thread leave no registers for a window
template <class E> __host__ __device__ constexpr int rs_look_win() { return sizeof(E) == 16 ? 8 : 1; }
// pairs per tile
template <class E> __host__ __device__ constexpr uint32_t rs_tile() { return kRsThreads * rs_items<E>(); }
inline uint32_t ntiles_of(uint64_t n) { return (uint32_t)((n + rs_tile<uint4>() - 1) / rs_tile<uint4>()); }

// Phase 1: pairs[i] = (key of record i, zero pad, i).  WORDS: records and
// the table are 4-byte aligned, so the key is read as ceil(key_bytes/4)
// words (never past the record: key_bytes <= rec, rec a multiple of 4).
// The digit counts of the first count_bytes key bytes (counts[j * 256 + d],
// zero on entry) are taken on the way, so the radix passes need not read the
// pairs for them.
template <bool WORDS>
__global__ void __launch_bounds__(256)
    k_extract_pairs(const uint8_t* __restrict__ src, uint64_t n, uint32_t rec, uint32_t key_bytes,
                    uint32_t count_bytes, uint4* __restrict__ pairs, uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[12 * 256];
  for (uint32_t x = threadIdx.x; x < count_bytes * 256; x += blockDim.x) h[x] = 0;
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
    for (uint32_t j = 0; j < count_bytes; ++j) atomicAdd(&h[j * 256 + ((w[j >> 2] >> (8 * (j & 3))) & 0xffu)], 1u);
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < count_bytes * 256; x += blockDim.x)
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

// Shared state of one CTA's tile in a radix pass.
struct RsShared {
  uint16_t whist[kRsWarps][256];  // pairs of digit d in warp w's share of the tile
  uint16_t wslot[kRsWarps][256];  // tile slot of warp w's first pair of digit d
  uint32_t s_base[256];           // output position of the pass's first pair of digit d
  uint32_t s_gpos[256];           // output position of this tile's first pair of digit d
  uint32_t s_toff[256];           // tile slot of this tile's first pair of digit d
  uint32_t s_wsum[8];
  uint32_t s_tile;
  int s_ok;
};

// Claim the CTA's next tile of a pass (its number in sh.s_tile) and clear
// the per-warp counts.
__device__ __forceinline__ uint32_t rs_claim(uint32_t* tile_ctr, RsShared& sh) {
  if (threadIdx.x == 0) sh.s_tile = atomicAdd(tile_ctr, 1u);
  for (uint32_t x = threadIdx.x; x < kRsWarps * 128; x += kRsThreads) reinterpret_cast<uint32_t*>(&sh.whist[0][0])[x] = 0;
  __syncthreads();
  return sh.s_tile;
}

// One tile t of a stable pass on key byte `byte` (tiles are numbered in the
// order CTAs claim them, so a tile only waits for tiles whose CTAs already
// run).  E: uint4 (16-byte pairs) or uint2 (8-byte pairs).  CG: the input was written
// earlier in the same launch, so it is read from L2 (ld.global.cg), never
// through a cache that may hold older lines.
template <class E, bool CG = false>
__device__ __forceinline__ void rs_tile_body(const E* __restrict__ in, E* __restrict__ out, uint64_t n, uint32_t byte,
                                             const uint32_t* __restrict__ digit_count, uint32_t* status, uint32_t t,
                                             int* err, long long wait_limit, RsShared& sh) {
  constexpr int kItems = rs_items<E>();
  constexpr uint32_t kTile = rs_tile<E>();
  static_assert(kTile <= 65536, "tile slots are 16-bit");
  extern __shared__ uint4 sraw[];
  E* sbuf = reinterpret_cast<E*>(sraw);  // kTile pairs
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
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
      sh.s_base[lane * 8 + j] = run;
      run += c[j];
    }
  }
  // this thread's pairs: kItems rounds of 32 consecutive pairs of its warp
  // (the digit is recomputed from the pair where it is needed)
  const uint64_t e0 = base + (uint64_t)warp * (32 * kItems) + lane;
  const uint32_t rem = n > e0 ? (n - e0 < kTile ? (uint32_t)(n - e0) : kTile) : 0u;  // item k valid: 32k < rem
  const E* __restrict__ inp = in + e0;
  E v[kItems];
  uint32_t rank2[kItems / 2];  // two 16-bit in-warp ranks per word (a rank is below the tile size)
  // all of the tile's loads first: the ranking below has warp barriers,
  // which would otherwise hold each load back until the previous round ends
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if ((uint32_t)k * 32 < rem) v[k] = CG ? __ldcg(inp + k * 32) : inp[k * 32];
  // stable in-warp ranks: round k's peers (valid lanes with the same digit)
  // are the AND of eight ballots, one per digit bit; the lane's rank is the
  // warp's count of that digit in earlier rounds plus its peers below it
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const bool ok = (uint32_t)k * 32 < rem;
    const uint32_t d = ok ? pair_digit(v[k], byte) : 0u;
    uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      peers &= __ballot_sync(0xffffffffu, bit != 0u) ^ (bit - 1u);
    }
    const uint32_t before = __popc(peers & lt);
    const uint32_t prior = ok ? sh.whist[warp][d] : 0u;
    __syncwarp();
    if (ok && before == 0) sh.whist[warp][d] = (uint16_t)(prior + __popc(peers));
    __syncwarp();
    if (k & 1) rank2[k >> 1] |= (prior + before) << 16;
    else rank2[k >> 1] = prior + before;
  }
  __syncthreads();
  const uint32_t dg = threadIdx.x & 255;
  uint32_t cnt = 0;  // the tile's count of digit dg
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) cnt += sh.whist[w][dg];
  if (threadIdx.x < 256) {
    // publish this tile's count of digit dg, then look back over earlier tiles
    volatile uint32_t* st = status;
    st[(uint64_t)t * 256 + dg] = (t == 0 ? kFlagPrefix : kFlagAgg) | cnt;
    uint32_t excl = 0;
    if (t > 0) {
      // tile j < t was claimed before this one, so its CTA is running and
      // publishes its count; the wait is bounded all the same.  The walk
      // reads kLookWin earlier tiles at a time (independent loads), then
      // sums them from the nearest down to the first inclusive prefix.
      constexpr int kLookWin = rs_look_win<E>();
      bool fin = false;
      for (int64_t j = (int64_t)t - 1; !fin && j >= 0; j -= kLookWin) {
        uint32_t w[kLookWin];
#pragma unroll
        for (int i = 0; i < kLookWin; ++i) w[i] = j - i >= 0 ? st[(uint64_t)(j - i) * 256 + dg] : 0u;
#pragma unroll
        for (int i = 0; i < kLookWin; ++i) {
          if (!fin && j - i >= 0) {
            uint32_t x = w[i];
            bool ok = true;
            if ((x & ~kCountMask) == 0)
              x = wait_word_bounded(status + (uint64_t)(j - i) * 256 + dg, wait_limit, &ok,
                                    [](uint32_t y) { return (y & ~kCountMask) != 0; });
            if (!ok) {
              atomicOr(err, ERR_TIMEOUT);
              fin = true;
            } else {
              excl += x & kCountMask;
              fin = (x & ~kCountMask) == kFlagPrefix;
            }
          }
        }
      }
      st[(uint64_t)t * 256 + dg] = kFlagPrefix | (excl + cnt);
    }
    sh.s_gpos[dg] = sh.s_base[dg] + excl;
  } else {
    // meanwhile the upper 256 threads lay out the tile: exclusive scan of the
    // counts over digits, then each warp's first slot per digit
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh.s_wsum[warp - 8] = x;
    asm volatile("bar.sync 1, 256;" ::: "memory");
    uint32_t off = x - cnt;
    for (int w = 0; w < warp - 8; ++w) off += sh.s_wsum[w];
    sh.s_toff[dg] = off;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      sh.wslot[w][dg] = (uint16_t)off;
      off += sh.whist[w][dg];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if ((uint32_t)k * 32 < rem) {
      const uint32_t d = pair_digit(v[k], byte);
      sbuf[sh.wslot[warp][d] + ((rank2[k >> 1] >> (16 * (k & 1))) & 0xffffu)] = v[k];
    }
  }
  __syncthreads();
  const uint32_t tn = (uint32_t)((n - base) < kTile ? (n - base) : kTile);
  for (uint32_t p = threadIdx.x; p < tn; p += kRsThreads) {
    const E q = sbuf[p];
    const uint32_t d = pair_digit(q, byte);
    out[(uint64_t)(uint32_t)(sh.s_gpos[d] + (p - sh.s_toff[d]))] = q;
  }
}

// One stable pass, one tile per CTA (the grid has a CTA per tile).
template <class E>
__global__ void __launch_bounds__(kRsThreads, kRsMinBlocks)
    k_rs_onesweep(const E* __restrict__ in, E* __restrict__ out, uint64_t n, uint32_t byte,
                  const uint32_t* __restrict__ digit_count, uint32_t* status, uint32_t* tile_ctr, int* err,
                  long long wait_limit) {
  __shared__ RsShared sh;
  const uint32_t t = rs_claim(tile_ctr, sh);
  rs_tile_body<E>(in, out, n, byte, digit_count, status, t, err, wait_limit, sh);
}

// Wait (bounded) until every CTA of the grid has arrived at barrier number
// `round` (counter *ctr, zero before the launch); false after the limit.
__device__ __forceinline__ bool grid_barrier(uint32_t* ctr, uint32_t round, long long limit, RsShared& sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    bool ok;
    const uint32_t target = round * gridDim.x;
    wait_word_bounded(ctr, limit, &ok, [target](uint32_t x) { return x >= target; });
    __threadfence();
    sh.s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return sh.s_ok != 0;
}

// The whole LSD sort (key bytes key_bytes-1 .. 0) of a[0 .. *n_dev) in one
// cooperative launch (every CTA resident): pass p reads a or b in turn,
// claims tiles from ctrs[p] and publishes into status region p % 2 (of
// region_words words each); a grid barrier (counter ctrs[key_bytes]) orders
// the clearing of region 0 before pass 0 and each pass before the next, and
// each pass clears the region the next one uses.  The result is in a for an
// even key_bytes, else in b.  counts: key_bytes x 256 digit counts; ctrs:
// key_bytes + 1 words, zero before the launch.  No pairs: the launch returns
// at once.
__global__ void __launch_bounds__(kRsThreads, kRsMinBlocks)
    k_rs_passes(uint4* a, uint4* b, const uint32_t* __restrict__ n_dev, uint32_t key_bytes,
                const uint32_t* __restrict__ counts, uint32_t* status, uint64_t region_words, uint32_t* ctrs,
                int* err, long long wait_limit) {
  __shared__ RsShared sh;
  const uint64_t n = *n_dev;
  const uint32_t ntiles = (uint32_t)((n + rs_tile<uint4>() - 1) / rs_tile<uint4>());
  if (ntiles == 0) return;
  for (uint64_t x = blockIdx.x * (uint64_t)kRsThreads + threadIdx.x; x < (uint64_t)ntiles * 256;
       x += (uint64_t)gridDim.x * kRsThreads)
    status[x] = 0;
  if (!grid_barrier(ctrs + key_bytes, 1, wait_limit, sh)) {
    if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
    return;
  }
  for (uint32_t p = 0; p < key_bytes; ++p) {
    const uint32_t byte = key_bytes - 1 - p;
    const uint4* in = (p & 1) ? b : a;
    uint4* out = (p & 1) ? a : b;
    uint32_t* region = status + (p & 1) * region_words;
    if (p + 1 < key_bytes) {  // the next pass's region: last used two passes ago
      uint32_t* next = status + ((p + 1) & 1) * region_words;
      for (uint64_t x = blockIdx.x * (uint64_t)kRsThreads + threadIdx.x; x < (uint64_t)ntiles * 256;
           x += (uint64_t)gridDim.x * kRsThreads)
        next[x] = 0;
    }
    for (;;) {
      const uint32_t t = rs_claim(ctrs + p, sh);
      if (t >= ntiles) break;
      rs_tile_body<uint4, true>(in, out, n, byte, counts + 256 * byte, region, t, err, wait_limit, sh);
      __syncthreads();
    }
    if (p + 1 < key_bytes && !grid_barrier(ctrs + key_bytes, p + 2, wait_limit, sh)) {
      if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
      return;
    }
  }
}

// ---- the bucket stage: after two LSD passes on key bytes 1 and 0 the pairs
// lie in 65,536 buckets of equal two-byte prefix, each in rid order; every
// bucket is then sorted on the rest of its key.

constexpr uint32_t kBuckets = 65536;
constexpr uint32_t kBucketMax = 256;  // the largest bucket a warp sorts itself
constexpr int kBsWarps = 8;

__device__ __forceinline__ uint32_t pair_prefix(const uint4& p) { return ((p.x & 0xffu) << 8) | ((p.x >> 8) & 0xffu); }

// off[b] = position of the first pair with prefix >= b (off[kBuckets] = n):
// each position i writes the buckets strictly after its predecessor's prefix
// up to its own (position n: up to kBuckets).
__global__ void __launch_bounds__(256) k_bucket_bounds(const uint4* __restrict__ pairs, uint64_t n,
                                                       uint32_t* __restrict__ off) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = i < n ? pair_prefix(pairs[i]) : kBuckets;
    const int64_t q = i > 0 ? (int64_t)pair_prefix(pairs[i - 1]) : -1;
    for (int64_t b = q + 1; b <= (int64_t)p; ++b) off[b] = (uint32_t)i;
  }
}

// Key bytes 3.. of a pair as big-endian words, then the rid: the order
// inside a run of equal first three key bytes.
__device__ __forceinline__ bool tail_greater(const uint4& a, const uint4& b) {
  const uint32_t a0 = __byte_perm(a.x, a.y, 0x3456), b0 = __byte_perm(b.x, b.y, 0x3456);
  if (a0 != b0) return a0 > b0;
  const uint32_t a1 = __byte_perm(a.y, a.z, 0x3456), b1 = __byte_perm(b.y, b.z, 0x3456);
  if (a1 != b1) return a1 > b1;
  if ((a.z >> 24) != (b.z >> 24)) return (a.z >> 24) > (b.z >> 24);
  return a.w > b.w;
}

constexpr uint32_t kRunMax = 32;  // the longest run of equal key byte 2 a lane sorts by insertion

// Each warp sorts whole buckets of up to kBucketMax pairs in place: a
// counting sort on key byte 2 in shared memory (the scatter order inside a
// digit does not matter), then each run of equal byte 2 sorted by insertion
// on the rest of the key and the rid, one lane per run.  A bucket larger
// than kBucketMax, or with a run longer than kRunMax, is appended whole (in
// its rid order) to big[] for the LSD fallback.
__global__ void __launch_bounds__(kBsWarps * 32) k_bucket_sort(uint4* __restrict__ pairs,
                                                               const uint32_t* __restrict__ off,
                                                               uint4* __restrict__ big, uint32_t* __restrict__ nbig) {
  __shared__ uint4 sk[kBsWarps][kBucketMax];
  __shared__ uint32_t sc[kBsWarps][256];
  constexpr int kPer = kBucketMax / 32;
  static_assert(kPer == 8, "the count layout holds 8 digits per lane");
  // digit d's count at ((d % 8) << 5) | (d / 8): lane l's digits 8l..8l+7 sit
  // in 8 different rows of one bank, so the per-lane scan is conflict-free
  auto ci = [](uint32_t d) { return ((d & 7u) << 5) | (d >> 3); };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint4* k = sk[warp];
  uint32_t* c = sc[warp];
  for (uint32_t b = blockIdx.x * kBsWarps + warp; b < kBuckets; b += gridDim.x * kBsWarps) {
    const uint32_t o = off[b], m = off[b + 1] - o;
    if (m <= 1) continue;
    bool to_big = m > kBucketMax;
    if (!to_big) {
      uint4 v[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) c[(q << 5) | lane] = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (lane + 32 * q < (int)m) v[q] = pairs[o + lane + 32 * q];
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (lane + 32 * q < (int)m) atomicAdd(&c[ci((v[q].x >> 16) & 0xffu)], 1u);
      __syncwarp();
      uint32_t cnt[kPer], sum = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        cnt[q] = c[(q << 5) | lane];
        sum += cnt[q];
      }
      uint32_t x = sum;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
        if (lane >= s) x += y;
      }
      uint32_t run = x - sum;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        c[(q << 5) | lane] = run;
        run += cnt[q];
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (lane + 32 * q < (int)m) k[atomicAdd(&c[ci((v[q].x >> 16) & 0xffu)], 1u)] = v[q];
      __syncwarp();
      // c[d] is now the end of digit d's run; runs of two or more are sorted
      bool too_long = false;
      uint32_t start = lane == 0 ? 0u : c[(7 << 5) | (lane - 1)];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const uint32_t end = c[(q << 5) | lane];
        if (end - start > kRunMax) {
          too_long = true;
        } else {
          for (uint32_t i = start + 1; i < end; ++i) {
            const uint4 t = k[i];
            uint32_t j = i;
            while (j > start && tail_greater(k[j - 1], t)) {
              k[j] = k[j - 1];
              --j;
            }
            k[j] = t;
          }
        }
        start = end;
      }
      to_big = __any_sync(0xffffffffu, too_long);
      __syncwarp();
      if (!to_big) {
        for (uint32_t i = lane; i < m; i += 32) pairs[o + i] = k[i];
        __syncwarp();
        continue;
      }
    }
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(nbig, m);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < m; i += 32) big[base + i] = pairs[o + i];
  }
}

// Digit counts of the first key_bytes bytes of big[0 .. *nbig).
__global__ void __launch_bounds__(256) k_count_big(const uint4* __restrict__ big, const uint32_t* __restrict__ nbig,
                                                   uint32_t key_bytes, uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[12 * 256];
  for (uint32_t x = threadIdx.x; x < key_bytes * 256; x += blockDim.x) h[x] = 0;
  __syncthreads();
  const uint64_t n = *nbig;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 p = big[i];
    const uint32_t w[3] = {p.x, p.y, p.z};
    for (uint32_t j = 0; j < key_bytes; ++j) atomicAdd(&h[j * 256 + ((w[j >> 2] >> (8 * (j & 3))) & 0xffu)], 1u);
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < key_bytes * 256; x += blockDim.x)
    if (h[x]) atomicAdd(&counts[x], h[x]);
}

// first[b] = position of the first pair of prefix b in the sorted fallback
// array (written only for the prefixes it holds).
__global__ void __launch_bounds__(256) k_big_first(const uint4* __restrict__ sorted, const uint32_t* __restrict__ nbig,
                                                   uint32_t* __restrict__ first) {
  const uint64_t n = *nbig;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = pair_prefix(sorted[j]);
    if (j == 0 || pair_prefix(sorted[j - 1]) != p) first[p] = (uint32_t)j;
  }
}

// The sorted fallback pairs back into their buckets' places: the j-th of
// them is the (j - first[b])-th pair of bucket b.
__global__ void __launch_bounds__(256) k_scatter_big(const uint4* __restrict__ sorted, const uint32_t* __restrict__ nbig,
                                                     const uint32_t* __restrict__ off,
                                                     const uint32_t* __restrict__ first, uint4* __restrict__ pairs) {
  const uint64_t n = *nbig;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 q = sorted[j];
    const uint32_t b = pair_prefix(q);
    pairs[(uint64_t)off[b] + (j - first[b])] = q;
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
  const size_t smem = rs_tile<E>() * sizeof(E);
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

// Words of the bucketed sort's state, all zeroed by one memset before the
// sort: the digit counts of key bytes 0 and 1, the two passes' tile
// counters, the fallback's pair count, its digit counts and its pass
// counters, then each of the two passes' status region.  After them: the
// fallback's two status regions (cleared by its own launch), the bucket
// offsets and the fallback's first position per prefix.
struct BucketState {
  static constexpr uint64_t kCounts = 0, kTileCtr = 3072, kNbig = 3136, kCountsBig = 3200, kCtrs = 6272,
                            kStatus = 6400;
  uint64_t region;  // words of one status region: 256 per tile
  explicit BucketState(uint64_t n) : region((uint64_t)ntiles_of(n) * 256) {}
  uint64_t zeroed() const { return kStatus + 2 * region; }
  uint64_t fstatus() const { return zeroed(); }
  uint64_t off() const { return fstatus() + 2 * region; }
  uint64_t first() const { return off() + kBuckets + 1; }
  uint64_t words() const { return first() + kBuckets; }
};

size_t sort_keyptr_tmp_bytes(uint64_t n, uint32_t key_bytes) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  if (key_bytes <= 2) return al(n * 16);
  return 2 * al(n * 16) + al(BucketState(n).words() * 4);
}

// Phases 1 and 2 of §3 into `pairs`.  Keys of at most two bytes: that many
// LSD passes.  Longer keys: two LSD passes on bytes 1 and 0 leave the pairs
// in buckets of equal two-byte prefix, each in rid order; every bucket of up
// to kBucketMax pairs is then sorted in place on key bytes 2.. and the rid
// (k_bucket_sort).  The pairs of the other buckets (ties, skewed keys) are
// appended, a bucket at a time, to one array that the full LSD sort orders
// (every key byte: its passes read the pair count on the device, so nothing
// waits for the host), and are then put back in their buckets' places.
int run_sort_keyptr(dpg_ctx& ctx, const uint8_t* src, uint64_t n, uint32_t rec, uint32_t key_bytes, uint8_t* pairs,
                    uint8_t* tmp, uint8_t* scan, cudaStream_t st) {
  if (n == 0) return DPG_OK;
  if (key_bytes == 0 || key_bytes > 12 || n > kCountMask) return DPG_EINVAL;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const bool buckets = key_bytes > 2;
  // keys of one or two bytes: an even number of passes ends where it started
  uint8_t* start = (!buckets && key_bytes % 2 == 1) ? tmp : pairs;
  uint8_t* other = start == pairs ? tmp : pairs;
  const uint32_t lsd_bytes = buckets ? 2u : key_bytes;
  const BucketState bs(n);
  uint32_t* state = reinterpret_cast<uint32_t*>(tmp + (buckets ? 2 * al(n * 16) : 0));
  uint32_t* counts = buckets ? state + BucketState::kCounts : radix_counts(scan);
  // the bucketed sort clears all of its small state and both passes' status
  // regions at once
  cudaError_t e = cudaMemsetAsync(counts, 0, buckets ? bs.zeroed() * 4 : 12 * 256 * 4, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  {
    TraceScope ts(ctx, "k_extract_pairs", st);
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx.sms * 8);
    if (rec % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 4 == 0)
      k_extract_pairs<true><<<grid, 256, 0, st>>>(src, n, rec, key_bytes, lsd_bytes, reinterpret_cast<uint4*>(start),
                                                  counts);
    else
      k_extract_pairs<false><<<grid, 256, 0, st>>>(src, n, rec, key_bytes, lsd_bytes, reinterpret_cast<uint4*>(start),
                                                   counts);
    ctx.launches++;
  }
  if (!buckets) {
    int status = DPG_OK;
    run_radix_pairs(ctx, start, other, scan, n, lsd_bytes, st, &status);
    return status;
  }

  uint4* p4 = reinterpret_cast<uint4*>(pairs);
  uint4* A = reinterpret_cast<uint4*>(tmp);
  uint4* C = reinterpret_cast<uint4*>(tmp + al(n * 16));
  {  // LSD passes on key bytes 1 and 0: pairs -> A -> pairs
    const size_t smem = rs_tile<uint4>() * sizeof(uint4);
    cudaFuncSetAttribute(k_rs_onesweep<uint4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int p = 0; p < 2; ++p) {
      TraceScope ts(ctx, "k_rs_onesweep", st);
      k_rs_onesweep<uint4><<<ntiles_of(n), kRsThreads, smem, st>>>(
          p == 0 ? p4 : A, p == 0 ? A : p4, n, 1u - p, counts + 256 * (1 - p), state + BucketState::kStatus + p * bs.region,
          state + BucketState::kTileCtr + p, ctx.d_err, ctx.wait_cycles);
      ctx.launches++;
    }
  }
  uint32_t* off = state + bs.off();
  uint32_t* nbig = state + BucketState::kNbig;
  uint32_t* first = state + bs.first();
  uint32_t* counts_big = state + BucketState::kCountsBig;
  const int grid = ctx.sms * 8;
  {
    TraceScope ts(ctx, "k_bucket_bounds", st);
    k_bucket_bounds<<<grid, 256, 0, st>>>(p4, n, off);
    ctx.launches++;
  }
  {
    TraceScope ts(ctx, "k_bucket_sort", st);
    k_bucket_sort<<<grid, kBsWarps * 32, 0, st>>>(p4, off, C, nbig);
    ctx.launches++;
  }
  // the fallback for the large buckets (no pairs at all for most keys)
  {
    TraceScope ts(ctx, "k_count_big", st);
    k_count_big<<<ctx.sms * 2, 256, 0, st>>>(C, nbig, key_bytes, counts_big);
    ctx.launches++;
  }
  // the LSD fallback in one cooperative launch (it returns at once when no
  // bucket needed it)
  const uint64_t region_words = bs.region;
  uint32_t* fstatus = state + bs.fstatus();
  uint32_t* ctrs = state + BucketState::kCtrs;
  const size_t smem = rs_tile<uint4>() * sizeof(uint4);
  int blocks_per_sm = 0;
  e = cudaFuncSetAttribute(k_rs_passes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_rs_passes, kRsThreads, smem);
  if (e == cudaSuccess && blocks_per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
  uint4* a = C;
  uint4* b = A;
  {
    TraceScope ts(ctx, "k_rs_passes", st);
    uint32_t kb = key_bytes;
    long long wl = ctx.wait_cycles;
    void* args[] = {&a, &b, &nbig, &kb, &counts_big, &fstatus, const_cast<uint64_t*>(&region_words), &ctrs,
                    &ctx.d_err, &wl};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_rs_passes), dim3(blocks_per_sm * ctx.sms),
                                    dim3(kRsThreads), args, smem, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cooperative launch");
    ctx.launches++;
  }
  if (key_bytes % 2 == 1) a = b;  // where the passes left the sorted pairs
  {
    TraceScope ts(ctx, "k_big_first", st);
    k_big_first<<<ctx.sms * 2, 256, 0, st>>>(a, nbig, first);
    ctx.launches++;
  }
  {
    TraceScope ts(ctx, "k_scatter_big", st);
    k_scatter_big<<<ctx.sms * 2, 256, 0, st>>>(a, nbig, off, first, p4);
    ctx.launches++;
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? DPG_OK : cuda_fail(ctx, e, "sort launch");
}

}  // namespace dpg
