// DPG record retrieval with runs held in the L2 (plan variant 4): Phase I
// partitions the rids into at most kL2MaxRuns runs of a few MB of source,
// Phase II probes each run while its source bytes are L2-resident, Phase III
// writes the destination in rid order (§2.1, Figure 1; run length: §2.1's
// L = half the cache, here the GPU's shared L2).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "dpg_device.cuh"
#include "dpg_internal.h"
#include "dpg_launch.cuh"

namespace dpg {
namespace {

constexpr int kRunsHistUnroll = 8;
constexpr int kRunsGatherThreads = 256;
constexpr int kRunsGatherUnroll = 8;
// k_probe_runs: 16-byte words per thread per chunk (128 B in flight; 8 against
// 4 measured 335 against 350 us at 32-byte records), and 3 CTAs per SM for
// the registers that takes.
constexpr int kProbeRunsU16 = 8;
constexpr int kProbeRunsMinCtas = 3;
// join rows (PK): half the words in flight at twice the CTAs per SM (the
// key check holds registers; at 64 registers the kernel ran at half the
// SM's warp slots)
constexpr int kProbeRunsU16Join = 4;
constexpr int kProbeRunsMinCtasJoin = 8;

// ------------------------------------------------------- L2-run plan (variant 4)
// The paper sizes a run to half the cache (Figure 1, L = CACHE_SIZE/2).  On
// GB300 the cache that all SMs share is the 126 MB L2, so this plan uses at most
// kL2MaxRuns runs of a few MB of source each.
//   Phase I  (k_hist_runs, k_part_runs): per CTA range the count of its
//            rids per run; run offsets (scanned by every k_part_runs CTA);
//            then each range is walked in tiles of T rids, a tile
//            counting-sorted by run in shared memory and written to the runs
//            as contiguous pieces at the range's cursors.  For Phase III each rid keeps either its place in its
//            sorted tile (2 bytes, plus the tile's count per run) or its place
//            in INTERNAL (a 4-byte slot).
//   Phase II (k_probe_runs below 64-byte records, the slot gather over run
//            order from 64 bytes): INTERNAL[k] = R[run_rid[k]]; the records
//            in flight fall in one or two runs, whose source bytes stay
//            L2-resident while they are probed.
//   Phase III (k_unpart_runs below 96-byte records): the mirror of Phase I.
//            A tile's entries of run b form one contiguous piece of INTERNAL
//            (at the range's cursor for b), so the tile reads its pieces with
//            coalesced loads into shared memory in sorted order and writes
//            the destination in rid order through the tile places.  From 96
//            bytes Phase III gathers through the slots; so do DPG-move join
//            rows, while DPG-sort join rows are rebuilt tile by tile like
//            records (fact rows up to 128 bytes), each followed by its
//            dimension row.

constexpr int kTileThreads = 512;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kPartIpt = 8;                        // Phase I tile: 4096 rids
constexpr uint32_t kUnpartStageMax = 64 * 1024;    // Phase III shared-memory records per tile
constexpr uint32_t kL2Ranges = 12;                 // Phase I / III CTA ranges per SM

// Exclusive scan of v[0, nb) into out[0, nb) by a block of kTileThreads
// (nb <= 2 * kTileThreads); wsum holds 32 words of scratch.
__device__ __forceinline__ void tile_scan(const uint32_t* v, uint32_t* out, uint32_t nb, uint32_t* wsum) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t x0 = 2 * threadIdx.x;
  const uint32_t v0 = x0 < nb ? v[x0] : 0u, v1 = x0 + 1 < nb ? v[x0 + 1] : 0u;
  uint32_t s = v0 + v1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= (uint32_t)o) s += y;
  }
  if (lane == 31) wsum[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < (uint32_t)kTileWarps ? wsum[lane] : 0u;
    uint32_t z = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= (uint32_t)o) z += y;
    }
    if (lane < (uint32_t)kTileWarps) wsum[lane] = z - w;
  }
  __syncthreads();
  const uint32_t e = wsum[warp] + s - v0 - v1;
  if (x0 < nb) out[x0] = e;
  if (x0 + 1 < nb) out[x0 + 1] = e + v0;
  __syncthreads();
}

// Phase I, pass 1 of the L2-run plan: for each CTA range g (a block takes
// ranges g = blockIdx.x, blockIdx.x + gridDim.x, ...) the count of its rids
// per run, added to the run total tot[b] (zero on entry) with one atomic whose
// old value, the range's offset inside run b, goes to cnt[g*nb + b]; the
// range check of every rid (before any destination write); strided rids
// copied out to `compact`.  Ranges take their places inside a run in the
// order of the atomics; Phase I and III both read them from cnt, and the
// result does not depend on that order.
template <class Rid>
__global__ void __launch_bounds__(kTileThreads, 4)
    k_hist_runs(Rid rid, uint64_t n, uint32_t n_src, uint32_t sl, uint32_t nb, uint32_t G, uint64_t per,
                uint32_t* __restrict__ cnt, uint32_t* __restrict__ tot, int* err, int32_t* __restrict__ compact) {
  extern __shared__ uint32_t h[];
  bool bad = false;
  for (uint32_t g = blockIdx.x; g < G; g += gridDim.x) {
    for (uint32_t b = threadIdx.x; b < nb; b += kTileThreads) h[b] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)g * per, hi = min(n, lo + per);
    for (uint64_t i0 = lo + threadIdx.x; i0 < hi; i0 += (uint64_t)kRunsHistUnroll * kTileThreads) {
      int32_t r[kRunsHistUnroll];
#pragma unroll
      for (int k = 0; k < kRunsHistUnroll; ++k) {
        const uint64_t i = i0 + (uint64_t)k * kTileThreads;
        r[k] = i < hi ? rid(i) : 0;
      }
#pragma unroll
      for (int k = 0; k < kRunsHistUnroll; ++k) {
        const uint64_t i = i0 + (uint64_t)k * kTileThreads;
        if (i < hi) {
          if (compact) compact[i] = r[k];
          if ((uint32_t)r[k] >= n_src) bad = true;
          else atomicAdd(&h[(uint32_t)r[k] >> sl], 1u);
        }
      }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += kTileThreads)
      cnt[(uint64_t)g * nb + b] = h[b] ? atomicAdd(&tot[b], h[b]) : 0u;
    __syncthreads();
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

// The same for an int32 rid array at a 16-byte-aligned address (no copy-out):
// the rids are read as 16-byte vectors of four (CTA ranges start at multiples
// of 4096 rids, so every range starts 16-byte aligned).
__global__ void __launch_bounds__(kTileThreads, 4)
    k_hist_runs4(const int32_t* __restrict__ rid, uint64_t n, uint32_t n_src, uint32_t sl, uint32_t nb, uint32_t G,
                 uint64_t per, uint32_t* __restrict__ cnt, uint32_t* __restrict__ tot, int* err) {
  extern __shared__ uint32_t h[];
  bool bad = false;
  auto count = [&](int32_t x) {
    if ((uint32_t)x >= n_src) bad = true;
    else atomicAdd(&h[(uint32_t)x >> sl], 1u);
  };
  for (uint32_t g = blockIdx.x; g < G; g += gridDim.x) {
    for (uint32_t b = threadIdx.x; b < nb; b += kTileThreads) h[b] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)g * per, hi = min(n, lo + per);
    const int4* r4 = reinterpret_cast<const int4*>(rid + lo);
    const uint32_t nv = (uint32_t)((hi - lo) >> 2);
    for (uint32_t v = threadIdx.x; v < nv; v += 2 * kTileThreads) {
      const int4 a = __ldg(r4 + v);
      const bool two = v + kTileThreads < nv;
      const int4 c = two ? __ldg(r4 + v + kTileThreads) : make_int4(0, 0, 0, 0);
      count(a.x);
      count(a.y);
      count(a.z);
      count(a.w);
      if (two) {
        count(c.x);
        count(c.y);
        count(c.z);
        count(c.w);
      }
    }
    for (uint64_t i = lo + 4 * (uint64_t)nv + threadIdx.x; i < hi; i += kTileThreads) count(__ldg(rid + i));
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += kTileThreads)
      cnt[(uint64_t)g * nb + b] = h[b] ? atomicAdd(&tot[b], h[b]) : 0u;
    __syncthreads();
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

// Phase I, pass 2 of the L2-run plan.  CTA g appends the rids of
// [g*per, (g+1)*per) to their runs at its cursors cur_g[g*nb + b], T rids at a
// time: the tile is counting-sorted by run in shared memory and written to the
// runs as contiguous pieces.  For Phase III it records either each rid's place
// in its sorted tile, tpos[i] (u16), and the tile's count of each run,
// tcnt_g[tile*nb + b] (u16), tile = i / T; or, with SLOT, each rid's place in
// INTERNAL, slot[i] (u32).
template <int IPT, bool SLOT>
__global__ void __launch_bounds__(kTileThreads, 3)
    k_part_runs(const int32_t* __restrict__ rid, uint64_t n, uint32_t sl, uint32_t nb, uint32_t G, uint64_t per,
                const uint32_t* __restrict__ tot, uint32_t* __restrict__ off, const uint32_t* __restrict__ cur_g,
                uint32_t* __restrict__ run_rid, uint16_t* __restrict__ tpos, uint16_t* __restrict__ tcnt_g,
                uint32_t* __restrict__ slot, const int* err) {
  constexpr uint32_t T = kTileThreads * IPT;
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ uint32_t wsum[32];
  if (__syncthreads_or(threadIdx.x == 0 && error_set(err))) return;
  uint32_t* cur = reinterpret_cast<uint32_t*>(sm);  // run b's next position in run_rid
  uint32_t* tcnt = cur + nb;
  uint32_t* toff = tcnt + nb;
  uint32_t* delta = toff + nb;                      // cur[b] - toff[b] for the tile
  uint32_t* runoff = delta + nb;                    // run b's first position in run_rid
  uint32_t* ent = runoff + nb;
  const uint32_t tid = threadIdx.x;
  // run offsets: exclusive scan of the run totals, in every CTA (block 0 also
  // stores them for Phase III)
  for (uint32_t x = tid; x < nb; x += kTileThreads) tcnt[x] = tot[x];
  __syncthreads();
  tile_scan(tcnt, runoff, nb, wsum);
  if (blockIdx.x == 0)
    for (uint32_t x = tid; x < nb; x += kTileThreads) off[x] = runoff[x];
  for (uint32_t g = blockIdx.x; g < G; g += gridDim.x) {
    for (uint32_t x = tid; x < nb; x += kTileThreads) {
      cur[x] = runoff[x] + cur_g[(uint64_t)g * nb + x];
      tcnt[x] = 0;
    }
    __syncthreads();
    const uint64_t lo = (uint64_t)g * per, hi = min(n, lo + per);
    uint32_t r[IPT];
    {
      const uint32_t m = (uint32_t)((hi - lo) < (uint64_t)T ? (hi - lo) : (uint64_t)T);
#pragma unroll
      for (int k = 0; k < IPT; ++k)
        r[k] = k * kTileThreads + tid < m ? (uint32_t)__ldg(rid + lo + k * kTileThreads + tid) : 0u;
    }
    for (uint64_t t0 = lo; t0 < hi; t0 += T) {
      const uint32_t tn = (uint32_t)((hi - t0) < (uint64_t)T ? (hi - t0) : (uint64_t)T);
      const bool full = tn == T;
      // next tile's rids, in flight meanwhile
      uint32_t rn[IPT], l[IPT];
      {
        const uint64_t t1 = t0 + T;
        const uint32_t m = t1 < hi ? (uint32_t)((hi - t1) < (uint64_t)T ? (hi - t1) : (uint64_t)T) : 0u;
        const int32_t* rt = rid + t1;
        if (m == T) {
#pragma unroll
          for (int k = 0; k < IPT; ++k) rn[k] = (uint32_t)__ldg(rt + k * kTileThreads + tid);
        } else {
#pragma unroll
          for (int k = 0; k < IPT; ++k)
            rn[k] = k * kTileThreads + tid < m ? (uint32_t)__ldg(rt + k * kTileThreads + tid) : 0u;
        }
      }
      // count, and each rid's rank among the tile's rids of its run
#pragma unroll
      for (int k = 0; k < IPT; ++k)
        if (full || k * kTileThreads + tid < tn) l[k] = atomicAdd(&tcnt[r[k] >> sl], 1u);
      __syncthreads();
      tile_scan(tcnt, toff, nb, wsum);
      uint16_t* tc = tcnt_g + (t0 / T) * nb;
      for (uint32_t x = tid; x < nb; x += kTileThreads) {
        const uint32_t c = tcnt[x];
        if (!SLOT) tc[x] = (uint16_t)c;
        delta[x] = cur[x] - toff[x];
        cur[x] += c;
        tcnt[x] = 0;
      }
      if (SLOT) __syncthreads();  // delta[] is read below
      uint16_t* tp = tpos + t0;
      uint32_t* sp = slot + t0;
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const uint32_t j = k * kTileThreads + tid;
        if (full || j < tn) {
          const uint32_t b = r[k] >> sl;
          const uint32_t p = toff[b] + l[k];
          ent[p] = r[k];
          if (SLOT) sp[j] = delta[b] + p;
          else tp[j] = (uint16_t)p;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const uint32_t q = k * kTileThreads + tid;
        if (full || q < tn) {
          const uint32_t rv = ent[q];
          run_rid[delta[rv >> sl] + q] = rv;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < IPT; ++k) r[k] = rn[k];
    }
  }
}

// Phase II of the L2-run plan for records under 64 bytes: INTERNAL[k] =
// R[run_rid[k]] for k in run order.  One resident wave of CTAs claims chunks
// of kRunsGatherThreads * U words in increasing k from *ctr, so the records
// probed at any time lie in one or two runs, which stay L2-resident.  The next
// chunk is claimed, and its rids loaded, while this chunk's source reads are
// in flight (one dependent round trip per chunk instead of two).
// (Larger records use the grid-stride gather over run order; having the L2
// prefetch the next run with cp.async.bulk.prefetch was measured slower:
// 590 against 442 us at 16 bytes.)
// PK (DPG-move join, §4.2.1): each probed dimension row must carry its own
// row number as the int64 little-endian key at byte pk_off; a row that does
// not raises the range bit before any output row is written.

template <int WB, bool PK>
__global__ void __launch_bounds__(kRunsGatherThreads, PK ? kProbeRunsMinCtasJoin : kProbeRunsMinCtas)
    k_probe_runs(const uint8_t* __restrict__ src, uint8_t* __restrict__ out, const uint32_t* __restrict__ run_rid,
                 uint64_t n, uint32_t W, FastDiv fdW, unsigned long long* ctr, int* err, uint32_t pk_off) {
  using T = typename WordT<WB>::T;
  constexpr int U = WB == 16 ? (PK ? kProbeRunsU16Join : kProbeRunsU16) : kRunsGatherUnroll;  // words per thread per chunk
  constexpr uint32_t CH = kRunsGatherThreads * U;
  __shared__ uint64_t s_c[2];
  if (error_set(err)) return;
  const T* s = reinterpret_cast<const T*>(src);
  T* d = reinterpret_cast<T*>(out);
  const uint64_t total = n * W;
  const uint64_t nch = (total + CH - 1) / CH;
  // rid of each of this thread's words of chunk c
  auto load_ids = [&](uint64_t c, uint32_t (&id)[U]) {
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint64_t t = c * CH + (uint64_t)k * kRunsGatherThreads + threadIdx.x;
      id[k] = (c < nch && t < total) ? __ldg(run_rid + fdiv(t, fdW)) : 0u;
    }
  };
  if (threadIdx.x == 0) s_c[0] = atomicAdd(ctr, 1ull);
  __syncthreads();
  uint64_t c = s_c[0];
  uint32_t id[U];
  load_ids(c, id);
  // The next chunk is claimed and its rids loaded while this chunk's source
  // reads are in flight.
  bool bad = false;
  const uint32_t pk_w0 = pk_off / WB, pk_w1 = (pk_off + 8 + WB - 1) / WB;
  for (int buf = 1; c < nch; buf ^= 1) {
    if (threadIdx.x == 0) s_c[buf] = atomicAdd(ctr, 1ull);
    const uint64_t base = c * CH + threadIdx.x;
    T v[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint64_t t = base + (uint64_t)k * kRunsGatherThreads;
      if (t < total) {
        const uint32_t w = (uint32_t)(t - fdiv(t, fdW) * W);
        // records: L2-resident run, no L1 fill (measured 400 against 407 us at
        // 16 B); join rows (PK): hot dimension rows repeat, and an L1 copy per
        // SM keeps their reads off the one L2 slice that holds them
        v[k] = PK ? __ldg(s + (uint64_t)id[k] * W + w) : __ldcg(s + (uint64_t)id[k] * W + w);
        if (PK && w >= pk_w0 && w < pk_w1 && !pk_word_ok<WB>(v[k], w, pk_off, id[k])) bad = true;
      }
    }
    __syncthreads();
    const uint64_t cn = s_c[buf];
    load_ids(cn, id);
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint64_t t = base + (uint64_t)k * kRunsGatherThreads;
      if (t < total) d[t] = v[k];
    }
    c = cn;
  }
  if (PK && bad) atomicOr(err, ERR_RANGE);
}

// Phase III of the L2-run plan: CTA g rebuilds dst[i] for i in
// [g*per, (g+1)*per) from INTERNAL, one Phase I tile at a time.  Run b's piece
// of the tile is contiguous in INTERNAL (at the CTA's cursor for b) and in the
// sorted tile (at toff[b]); a warp copies one piece at a time.  The next
// tile's tpos and counts are loaded while the current tile is copied.
// STAGE: pieces are copied into shared memory in sorted order (cp.async when
// WB >= 4), then dst[t0 + j] = stage[tpos[t0 + j]] is written in rid order, as
// 16-byte vectors when VEC (WB = 4 or 8, 16-byte-aligned destination).
// Without STAGE (large records) each sorted entry is copied straight to its
// destination record through the inverse of tpos.
// JOIN (DPG-sort join rows, §4.2.1): the destination row of tile entry j is
// the staged fact row || dimension row fk, fk the int32 at byte fk_off of
// that staged fact row (the key it was sorted by); the int64 little-endian
// key at byte pk_off of the dimension row must equal fk, else the range bit.
// Rows are written as one word stream.
struct JoinTail {
  const uint8_t* dim;
  uint32_t wd;  // dimension-row words
  uint32_t fk_off;
  uint32_t pk_off;
  FastDiv fd_row;  // fact-row words + wd
};
// join-row words in flight per thread (2: 4.77 ms on the 2e8-row join, 4:
// 5.05 ms, 8: 5.93 ms); the join tile runs two CTAs per SM (64 registers;
// unbounded it takes 80 and one CTA).  The record tiles stay unbounded: an
// explicit minimum of one CTA lets the compiler take up to 79 registers
// where it otherwise takes 32-60.
constexpr int kJoinUnroll = 2;

template <int WB, int IPT, bool STAGE, bool VEC, bool JOIN = false>
__global__ void __launch_bounds__(kTileThreads, JOIN ? 2 : 0)
    k_unpart_runs(uint64_t n, uint32_t nb, uint32_t G, uint64_t per, const uint32_t* __restrict__ off,
                  const uint32_t* __restrict__ cur_g, const uint16_t* __restrict__ tpos,
                  const uint16_t* __restrict__ tcnt_g, const uint8_t* __restrict__ internal,
                  uint8_t* __restrict__ dst, uint32_t W, FastDiv fdW, int* err, JoinTail jt) {
  using Wd = typename WordT<WB>::T;
  static_assert(!JOIN || (STAGE && !VEC), "join rows are staged word streams");
  constexpr uint32_t T = kTileThreads * IPT;
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ uint32_t wsum[32];
  if (__syncthreads_or(threadIdx.x == 0 && error_set(err))) return;
  uint32_t* base = reinterpret_cast<uint32_t*>(sm);  // INTERNAL position of the tile's piece of run b
  uint32_t* tcnt = base + nb;
  uint32_t* toff = tcnt + nb;
  uint16_t* pos = reinterpret_cast<uint16_t*>(sm + (((size_t)nb * 12 + 15) & ~size_t(15)));  // tpos, or its inverse
  Wd* stage = reinterpret_cast<Wd*>(reinterpret_cast<uint8_t*>(pos) + 2 * T);
  const Wd* iw = reinterpret_cast<const Wd*>(internal);
  Wd* dw = reinterpret_cast<Wd*>(dst);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool bad = false;
  // this thread owns runs x0 and x0 + 1: their cursors live in registers
  const uint32_t x0 = 2 * threadIdx.x;
  for (uint32_t g = blockIdx.x; g < G; g += gridDim.x) {
  uint32_t cur0 = x0 < nb ? off[x0] + cur_g[(uint64_t)g * nb + x0] : 0u;
  uint32_t cur1 = x0 + 1 < nb ? off[x0 + 1] + cur_g[(uint64_t)g * nb + x0 + 1] : 0u;
  const uint64_t lo = (uint64_t)g * per, hi = min(n, lo + per);
  uint32_t tp[IPT], c0, c1;
  auto fetch = [&](uint64_t t0) {
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const uint64_t i = t0 + k * kTileThreads + threadIdx.x;
      tp[k] = i < hi ? (uint32_t)tpos[i] : 0u;
    }
    const uint16_t* tc = tcnt_g + (t0 / T) * nb;
    const bool in = t0 < hi;
    c0 = in && x0 < nb ? (uint32_t)tc[x0] : 0u;
    c1 = in && x0 + 1 < nb ? (uint32_t)tc[x0 + 1] : 0u;
  };
  fetch(lo);
  for (uint64_t t0 = lo; t0 < hi; t0 += T) {
    const uint32_t tn = (uint32_t)((hi - t0) < (uint64_t)T ? (hi - t0) : (uint64_t)T);
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const uint32_t j = k * kTileThreads + threadIdx.x;
      if (j < tn) {
        if (STAGE) pos[j] = (uint16_t)tp[k];
        else pos[tp[k]] = (uint16_t)j;
      }
    }
    // exclusive scan of the tile's counts; cursors advance past the tile
    {
      uint32_t s = c0 + c1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= (uint32_t)o) s += y;
      }
      if (lane == 31) wsum[warp] = s;
      __syncthreads();
      if (warp == 0) {
        const uint32_t w = lane < (uint32_t)kTileWarps ? wsum[lane] : 0u;
        uint32_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
          if (lane >= (uint32_t)o) z += y;
        }
        if (lane < (uint32_t)kTileWarps) wsum[lane] = z - w;
      }
      __syncthreads();
      const uint32_t e = wsum[warp] + s - c0 - c1;
      if (x0 < nb) {
        toff[x0] = e;
        tcnt[x0] = c0;
        base[x0] = cur0;
        cur0 += c0;
      }
      if (x0 + 1 < nb) {
        toff[x0 + 1] = e + c0;
        tcnt[x0 + 1] = c1;
        base[x0 + 1] = cur1;
        cur1 += c1;
      }
    }
    fetch(t0 + T);  // next tile, in flight meanwhile
    __syncthreads();
    Wd* d0 = dw + t0 * W;
    if constexpr (STAGE) {
      for (uint32_t b = warp; b < nb; b += kTileWarps) {
        const uint32_t c = tcnt[b] * W;
        const Wd* g = iw + (uint64_t)base[b] * W;
        Wd* s = stage + toff[b] * W;
        if constexpr (WB >= 4) {
          for (uint32_t u = lane; u < c; u += 32) cp_async<WB>(s + u, g + u);
        } else {
          for (uint32_t u = lane; u < c; u += 32) s[u] = g[u];
        }
      }
      if constexpr (WB >= 4) cp_async_wait_all();
      __syncthreads();
      const uint32_t total = tn * W;
      if constexpr (JOIN) {
        const uint32_t row_w = W + jt.wd, rows_w = tn * row_w;
        const uint32_t pk_w0 = jt.pk_off / WB, pk_w1 = (jt.pk_off + 8 + WB - 1) / WB;
        const Wd* dimw = reinterpret_cast<const Wd*>(jt.dim);
        const uint8_t* sfk = reinterpret_cast<const uint8_t*>(stage) + jt.fk_off;  // fk_off % 4 == 0
        Wd* o0 = dw + t0 * row_w;
        // word u = row j, word w of the row, walked in steps of kTileThreads words
        const uint32_t qs = (uint32_t)fdiv(kTileThreads, jt.fd_row), rs = kTileThreads - qs * row_w;
        uint32_t j = (uint32_t)fdiv(threadIdx.x, jt.fd_row), w = threadIdx.x - j * row_w;
        for (uint32_t t = threadIdx.x; t < rows_w; t += kTileThreads * kJoinUnroll) {
          Wd x[kJoinUnroll];
#pragma unroll
          for (int k = 0; k < kJoinUnroll; ++k) {
            const uint32_t u = t + k * kTileThreads;
            if (u < rows_w) {
              if (w < W) {
                x[k] = stage[(uint32_t)pos[j] * W + w];
              } else {
                const uint32_t key = *reinterpret_cast<const uint32_t*>(sfk + (uint32_t)pos[j] * (W * WB));
                const uint32_t wd = w - W;
                x[k] = dimw[(uint64_t)key * jt.wd + wd];
                if (wd >= pk_w0 && wd < pk_w1 && !pk_word_ok<WB>(x[k], wd, jt.pk_off, key)) bad = true;
              }
            }
            j += qs;
            w += rs;
            if (w >= row_w) {
              w -= row_w;
              ++j;
            }
          }
#pragma unroll
          for (int k = 0; k < kJoinUnroll; ++k) {
            const uint32_t u = t + k * kTileThreads;
            if (u < rows_w) o0[u] = x[k];
          }
        }
      } else if constexpr (VEC) {
        // 16-byte chunk c = words [V*c, V*c + V) of the tile's destination
        constexpr uint32_t V = 16 / WB;
        const uint32_t C = total / V;
        uint4* dv = reinterpret_cast<uint4*>(d0);
        for (uint32_t c = threadIdx.x; c < C; c += kTileThreads) {
          const uint32_t t = c * V;
          uint32_t j = (uint32_t)fdiv(t, fdW), w = t - j * W;
          Wd x[V];
#pragma unroll
          for (uint32_t k = 0; k < V; ++k) {
            x[k] = stage[(uint32_t)pos[j] * W + w];
            if (++w == W) {
              w = 0;
              ++j;
            }
          }
          if constexpr (WB == 4) dv[c] = make_uint4(x[0], x[1], x[2], x[3]);
          else dv[c] = make_uint4(x[0].x, x[0].y, x[1].x, x[1].y);
        }
        for (uint32_t t = C * V + threadIdx.x; t < total; t += kTileThreads) {
          const uint32_t j = (uint32_t)fdiv(t, fdW), w = t - j * W;
          d0[t] = stage[(uint32_t)pos[j] * W + w];
        }
      } else {
        for (uint32_t t = threadIdx.x; t < total; t += kTileThreads) {
          const uint32_t j = (uint32_t)fdiv(t, fdW), w = t - j * W;
          d0[t] = stage[(uint32_t)pos[j] * W + w];
        }
      }
    } else {
      // pos[] holds the inverse: sorted entry q belongs to tile rid pos[q]
      for (uint32_t b = warp; b < nb; b += kTileWarps) {
        const uint32_t c = tcnt[b] * W;
        const Wd* g = iw + (uint64_t)base[b] * W;
        const uint32_t q0 = toff[b];
        for (uint32_t u = lane; u < c; u += 32) {
          const uint32_t q = (uint32_t)fdiv(u, fdW), w = u - q * W;
          d0[(uint64_t)pos[q0 + q] * W + w] = g[u];
        }
      }
    }
    __syncthreads();
  }
  }
  if (JOIN && bad) atomicOr(err, ERR_RANGE);
}


// ------------------------------------------------------------------ host side

// Variant 4 (L2 runs): k_hist_runs -> k_part_runs -> k_probe_l2
// (Phase II gather in run order) -> k_unpart_runs.
struct Layout4 {
  uint32_t sl, nb, G, T;
  uint64_t per, tiles;
  bool stage_mode, slot_mode, strided;
  size_t b_cnt, b_tot, b_off, b_ctr, b_run, b_tpos, b_tcnt, b_rc, b_stage, need;
};

// Tile of the L2-run plan (Phase I and III): the largest power of two up to
// 4096 rids whose records fit kUnpartStageMax bytes of shared memory (at least
// 512 rids); larger records are not staged, 2048 rids per tile.
inline void part_tile(uint32_t rec, uint32_t& T, bool& stage) {
  const uint64_t smax = (uint64_t)env_int("DPG_UNPART_STAGE_MAX", (int)kUnpartStageMax);
  T = kTileThreads * kPartIpt;
  while (T > (uint32_t)kTileThreads && (uint64_t)T * rec > smax) T >>= 1;
  stage = (uint64_t)T * rec <= smax;
  if (!stage) T = 2048;
}

Layout4 layout4(const dpg_ctx& ctx, const Retrieval& r, const Plan& plan, bool strided) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  Layout4 L;
  L.sl = (uint32_t)plan.seg_log2;
  L.nb = (uint32_t)((r.n_src + (1ull << L.sl) - 1) >> L.sl);
  // Phase III: records of 96 bytes and more are gathered through a 4-byte
  // INTERNAL slot per rid (the 3-pass gather), so Phase I takes its largest
  // tile; smaller ones are rebuilt tile by tile from 2-byte tile places
  // DPG-sort join rows are rebuilt like records where the fact rows can be
  // staged (up to 128 bytes, the smallest tile's share); other join rows go
  // through slots
  const bool join_tiles = r.join && r.join->mode == 1 && r.rec <= 128;
  L.slot_mode = env_int("DPG_L2_SLOT", r.join ? !join_tiles : r.rec >= 96) != 0 || (r.join && !join_tiles);
  part_tile(L.slot_mode ? 1 : r.rec, L.T, L.stage_mode);
  // CTA ranges: whole 4096-rid blocks (every tile starts at a multiple of T),
  // kL2Ranges per SM so that every resident count of 2, 3 or 4 CTAs per SM
  // takes the same number of ranges
  const uint64_t block = (uint64_t)kTileThreads * kPartIpt;
  const uint64_t g_max = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)ctx.sms * kL2Ranges,
                                                                  (r.n + block - 1) / block));
  L.per = ((r.n + g_max - 1) / g_max + block - 1) / block * block;
  L.G = (uint32_t)((r.n + L.per - 1) / L.per);
  L.tiles = (r.n + L.T - 1) / L.T;
  L.strided = strided;
  L.b_cnt = al((size_t)L.nb * L.G * 4);
  L.b_tot = al((size_t)L.nb * 4);
  L.b_off = al(((size_t)L.nb + 1) * 4);
  L.b_ctr = 256;
  L.b_run = al(r.n * 4);
  L.b_tpos = al(r.n * (L.slot_mode ? 4 : 2));
  L.b_tcnt = L.slot_mode ? 0 : al((size_t)L.tiles * L.nb * 2);
  L.b_rc = strided ? al(r.n * 4) : 0;
  L.b_stage = al(r.n * r.rec);
  L.need = L.b_cnt + L.b_tot + L.b_off + L.b_ctr + L.b_run + L.b_tpos + L.b_tcnt + L.b_rc + L.b_stage;
  return L;
}

template <int WB, bool VEC>
void launch_unpart(dpg_ctx& ctx, const Layout4& L, uint64_t n, uint32_t rec, const uint32_t* off,
                   const uint32_t* cnt, const uint16_t* tpos, const uint16_t* tcnt, const uint8_t* internal,
                   uint8_t* dst, cudaStream_t st) {
  const uint32_t W = rec / WB;
  const FastDiv f = make_fastdiv(W);
  const size_t smem = (((size_t)L.nb * 12 + 15) & ~size_t(15)) + 2 * (size_t)L.T +
                      (L.stage_mode ? (size_t)L.T * rec : 0);
#define DPG_UNPART(IPTV, STG)                                                                                  \
  {                                                                                                            \
    auto kern = k_unpart_runs<WB, IPTV, STG, VEC && STG>;                                                      \
    set_smem(kern, smem);                                                                                      \
    const uint32_t grid = std::min<uint32_t>(L.G, ctx.sms * resident_per_sm(kern, kTileThreads, smem));        \
    kern<<<grid, kTileThreads, smem, st>>>(n, L.nb, L.G, L.per, off, cnt, tpos, tcnt, internal, dst, W, f,     \
                                           ctx.d_err, JoinTail{});                                             \
  }
  if (!L.stage_mode) DPG_UNPART(4, false)
  else if (L.T == 4096) DPG_UNPART(8, true)
  else if (L.T == 2048) DPG_UNPART(4, true)
  else if (L.T == 1024) DPG_UNPART(2, true)
  else DPG_UNPART(1, true)
#undef DPG_UNPART
}

// Phase III of the DPG-sort join on this plan: k_unpart_runs<JOIN> writes
// fact row || dimension row per tile entry (fact rows staged, see part_tile;
// the dimension row is the one the staged row's foreign key names).
template <int WB>
void launch_unpart_join(dpg_ctx& ctx, const Layout4& L, const Retrieval& r, const uint32_t* off, const uint32_t* cnt,
                        const uint16_t* tpos, const uint16_t* tcnt, const uint8_t* internal) {
  const JoinSpec& j = *r.join;
  const uint32_t W = r.rec / WB;
  const FastDiv f = make_fastdiv(W);
  const JoinTail jt{j.dim, j.dim_bytes / WB, j.fk_off, j.pk_off, make_fastdiv(W + j.dim_bytes / WB)};
  const size_t smem = (((size_t)L.nb * 12 + 15) & ~size_t(15)) + 2 * (size_t)L.T + (size_t)L.T * r.rec;
#define DPG_UNPART_JOIN(IPTV)                                                                                 \
  {                                                                                                           \
    auto kern = k_unpart_runs<WB, IPTV, true, false, true>;                                                   \
    set_smem(kern, smem);                                                                                     \
    const uint32_t grid = std::min<uint32_t>(L.G, ctx.sms * resident_per_sm(kern, kTileThreads, smem));       \
    kern<<<grid, kTileThreads, smem, r.stream>>>(r.n, L.nb, L.G, L.per, off, cnt, tpos, tcnt, internal, j.out, \
                                                 W, f, ctx.d_err, jt);                                        \
  }
  if (L.T == 4096) DPG_UNPART_JOIN(8)
  else if (L.T == 2048) DPG_UNPART_JOIN(4)
  else if (L.T == 1024) DPG_UNPART_JOIN(2)
  else DPG_UNPART_JOIN(1)
#undef DPG_UNPART_JOIN
}

template <class Rid>
int run_dpg_l2_t(dpg_ctx& ctx, const Retrieval& r, Rid rid, const Plan& plan) {
  const bool strided = !std::is_same<Rid, RidArray>::value;
  const Layout4 L = layout4(ctx, r, plan, strided);
  const uint32_t sl = L.sl, nb = L.nb, G = L.G;
  if (nb > kL2MaxRuns) return DPG_EINVAL;
  if (int s = ensure_scratch(ctx, L.need)) return s;
  uint8_t* p = static_cast<uint8_t*>(ctx.scratch);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(p); p += L.b_cnt;
  uint32_t* tot = reinterpret_cast<uint32_t*>(p); p += L.b_tot;
  uint32_t* off = reinterpret_cast<uint32_t*>(p); p += L.b_off;
  unsigned long long* pctr = reinterpret_cast<unsigned long long*>(p); p += L.b_ctr;
  uint32_t* run_rid = reinterpret_cast<uint32_t*>(p); p += L.b_run;
  uint16_t* tpos = reinterpret_cast<uint16_t*>(p);
  uint32_t* slot = reinterpret_cast<uint32_t*>(p);  // the same piece in slot mode
  p += L.b_tpos;
  uint16_t* tcnt = reinterpret_cast<uint16_t*>(p); p += L.b_tcnt;
  int32_t* rc = strided ? reinterpret_cast<int32_t*>(p) : nullptr; p += L.b_rc;
  uint8_t* stage = p;
  cudaError_t e = cudaMemsetAsync(tot, 0, (size_t)nb * 4, r.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(pctr, 0, 8, r.stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  {
    TraceScope ts(ctx, "k_hist_runs", r.stream);
    const size_t smem = (size_t)nb * 4;
    if (!strided && reinterpret_cast<uintptr_t>(r.rids.base) % 16 == 0) {
      set_smem(k_hist_runs4, smem);
      const uint32_t grid = std::min<uint32_t>(G, ctx.sms * resident_per_sm(k_hist_runs4, kTileThreads, smem));
      k_hist_runs4<<<grid, kTileThreads, smem, r.stream>>>(reinterpret_cast<const int32_t*>(r.rids.base), r.n,
                                                           (uint32_t)r.n_src, sl, nb, G, L.per, cnt, tot, ctx.d_err);
    } else {
      auto kern = k_hist_runs<Rid>;
      set_smem(kern, smem);
      const uint32_t grid = std::min<uint32_t>(G, ctx.sms * resident_per_sm(kern, kTileThreads, smem));
      kern<<<grid, kTileThreads, smem, r.stream>>>(rid, r.n, (uint32_t)r.n_src, sl, nb, G, L.per, cnt, tot,
                                                   ctx.d_err, rc);
    }
  }
  const int32_t* ra = strided ? rc : reinterpret_cast<const int32_t*>(r.rids.base);
  {
    TraceScope ts(ctx, "k_part_runs", r.stream);
    const size_t smem = (size_t)nb * 20 + (size_t)L.T * 4;  // cur, tcnt, toff, delta, runoff, ent
#define DPG_PART(IPTV)                                                                                          \
  {                                                                                                             \
    auto kern = L.slot_mode ? k_part_runs<IPTV, true> : k_part_runs<IPTV, false>;                               \
    set_smem(kern, smem);                                                                                       \
    const uint32_t grid = std::min<uint32_t>(G, ctx.sms * resident_per_sm(kern, kTileThreads, smem));           \
    kern<<<grid, kTileThreads, smem, r.stream>>>(ra, r.n, sl, nb, G, L.per, tot, off, cnt, run_rid, tpos, tcnt, \
                                                 slot, ctx.d_err);                                              \
  }
    if (L.T == 4096) DPG_PART(8)
    else if (L.T == 2048) DPG_PART(4)
    else if (L.T == 1024) DPG_PART(2)
    else DPG_PART(1)
#undef DPG_PART
  }
  ctx.launches += 2;  // k_hist_runs, k_part_runs
  // Phase II: INTERNAL[k] = R[run_rid[k]], k in run order
  const uint32_t wb2 = std::min(pow2_align(r.rec), pow2_align(reinterpret_cast<uintptr_t>(r.src)));
  const bool pk = r.join && r.join->mode == 0;
  if (r.rec >= 64 && !pk) {
    launch_slot_gather(ctx, wb2, r.src, stage, run_rid, r.n, r.rec, (uint32_t)r.n_src, r.stream, "k_probe_l2");
  } else {
    TraceScope ts(ctx, "k_probe_l2", r.stream);
    const uint32_t W = r.rec / wb2;
    const FastDiv f = make_fastdiv(W);
    const uint32_t pk_off = pk ? r.join->pk_off : 0u;
#define DPG_PR(WBV)                                                                                              \
  {                                                                                                              \
    auto kern = pk ? k_probe_runs<WBV, true> : k_probe_runs<WBV, false>;                                         \
    const uint32_t grid = ctx.sms * resident_per_sm(kern, kRunsGatherThreads, 0);                                \
    kern<<<grid, kRunsGatherThreads, 0, r.stream>>>(r.src, stage, run_rid, r.n, W, f, pctr, ctx.d_err, pk_off);  \
  }
    switch (wb2) {
      case 16: DPG_PR(16) break;
      case 8: DPG_PR(8) break;
      case 4: DPG_PR(4) break;
      case 2: DPG_PR(2) break;
      default: DPG_PR(1) break;
    }
#undef DPG_PR
    ctx.launches++;
  }
  // Phase III
  if (r.join && !L.slot_mode) {
    TraceScope ts(ctx, "k_unpart_join", r.stream);
    const JoinSpec& j = *r.join;
    const uint32_t wb3 = std::min({pow2_align(r.rec), pow2_align(j.dim_bytes),
                                   pow2_align(reinterpret_cast<uintptr_t>(j.out)),
                                   pow2_align(reinterpret_cast<uintptr_t>(j.dim))});
    switch (wb3) {
      case 16: launch_unpart_join<16>(ctx, L, r, off, cnt, tpos, tcnt, stage); break;
      case 8: launch_unpart_join<8>(ctx, L, r, off, cnt, tpos, tcnt, stage); break;
      case 4: launch_unpart_join<4>(ctx, L, r, off, cnt, tpos, tcnt, stage); break;
      case 2: launch_unpart_join<2>(ctx, L, r, off, cnt, tpos, tcnt, stage); break;
      default: launch_unpart_join<1>(ctx, L, r, off, cnt, tpos, tcnt, stage); break;
    }
    ctx.launches++;
  } else if (r.join) {
    launch_join_phase3(ctx, r, stage, slot);
  } else if (L.slot_mode) {
    const uint32_t wb3 = std::min(pow2_align(r.rec), pow2_align(reinterpret_cast<uintptr_t>(r.dst)));
    launch_slot_gather(ctx, wb3, stage, r.dst, slot, r.n, r.rec, (uint32_t)r.n_src, r.stream, "k_gather_phase3");
  } else {
    TraceScope ts(ctx, "k_unpart_runs", r.stream);
    const uint32_t wb3 = std::min(pow2_align(r.rec), pow2_align(reinterpret_cast<uintptr_t>(r.dst)));
    // 16-byte destination vectors: every tile starts at a multiple of 512
    // rids, so at a 16-byte boundary of a 16-byte-aligned destination
    const bool vec = pow2_align(reinterpret_cast<uintptr_t>(r.dst)) == 16 && r.rec >= 16;
#define DPG_UNP(WBV, V) launch_unpart<WBV, V>(ctx, L, r.n, r.rec, off, cnt, tpos, tcnt, stage, r.dst, r.stream)
    switch (wb3) {
      case 16: DPG_UNP(16, false); break;
      case 8:
        if (vec) DPG_UNP(8, true);
        else DPG_UNP(8, false);
        break;
      case 4:
        if (vec) DPG_UNP(4, true);
        else DPG_UNP(4, false);
        break;
      case 2: DPG_UNP(2, false); break;
      default: DPG_UNP(1, false); break;
    }
#undef DPG_UNP
    ctx.launches++;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "dpg l2 launch");
  return DPG_OK;
}

}  // namespace

int run_dpg_l2(dpg_ctx& ctx, const Retrieval& r, const Plan& plan) {
  if (r.rids.stride == 4)
    return run_dpg_l2_t<RidArray>(ctx, r, RidArray{reinterpret_cast<const int32_t*>(r.rids.base)}, plan);
  return run_dpg_l2_t<RidStrided>(ctx, r, RidStrided{r.rids.base, r.rids.stride}, plan);
}

size_t l2_scratch_need(const dpg_ctx& ctx, const Retrieval& r, const Plan& plan, bool strided) {
  return layout4(ctx, r, plan, strided).need;
}

}  // namespace dpg
