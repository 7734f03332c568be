// The batch executor: a whole batch of record retrievals and DPG-move joins
// run by persistent kernels over a device table of work items (dpg_run_batch
// and dpg_retrieve_batch in include/dpg.h): persistent launches per DPG
// phase, each claiming that phase's items of its groups, or (fused) all
// phases in one persistent launch.  Phases C and D are split by the groups'
// word size and plan: the common groups (slot plan, 4-, 8- or 16-byte words;
// for phase C also the scatter plan's 16-byte words) run in the lean
// k_exec_cd16, one instantiation each, at four CTAs per SM; the rest runs in
// the generic k_exec, whose one register allocation for every word size,
// plan and join leaves it two CTAs per SM.
//
// Requests that read the same source table with the same record size form a
// group (a join is a group of its own: its source is the dimension table,
// its rids the fact table's foreign-key column).  A group is retrieved by
// distribute-probe-gather (§2.1) with runs of a few MB held in the L2:
//   phase A  per range of kExRange group rids: each rid checked against its
//            own request's n_src, counted per run in shared memory; one
//            atomic per (range, run) claims the range's place in the run.
//            Rids of requests that are not laid out back to back in one
//            array are copied out in group order on the way.
//   phase B  per range: the run offsets (a scan of the run totals), then
//            tiles of kExTile rids counting-sorted by run in shared memory;
//            the run-ordered rids are written as one contiguous piece per
//            (tile, run), and per rid either its INTERNAL slot (slot plan) or,
//            per run position, the address of its destination record
//            (scatter plan).
//   phase C  per item of kExItemBytes of words in run order: the records of one or
//            two L2-resident runs copied to INTERNAL (slot plan; a join checks
//            each dimension row's key on the way) or straight to their
//            destination records (scatter plan, Phases II and III fused).
//   phase D  (slot plan) per item of kExItemBytes of destination words: dst[i] =
//            INTERNAL[slot[i]], or the join row fact[i] || INTERNAL[slot[i]].
// The items are laid out phase by phase (every group's A items, then every
// group's B items, ...).  In the fused launch CTAs claim them in that order
// from one counter, so an item only ever waits for items claimed before it,
// whose CTAs are already running: the executor cannot deadlock.  Every
// phase-B item waits for all phase-A items of the batch (so a bad rid
// anywhere leaves every destination untouched); C and D wait for their
// group's previous phase.  Each wait is bounded by the context's wait limit
// and gives up with the timeout bit set.  The phase launches need no waits
// (each follows the previous one on the stream) and each runs at its own
// occupancy: the fused kernel's register budget is the largest phase's, which
// leaves the memory-bound phases C and D with too few warps in flight
// (measured on 1e9-byte retrievals: 1.79 against 1.57 ms at 16-byte records,
// 0.70 against 0.53 ms at 256 bytes).
#include <algorithm>
#include <cstring>
#include <vector>

#include "dpg_device.cuh"
#include "dpg_internal.h"
#include "dpg_launch.cuh"

namespace dpg {
namespace {

constexpr int kExThreads = 512;
constexpr int kExWarps = kExThreads / 32;
constexpr int kExIpt = 8;
constexpr uint32_t kExTile = kExThreads * kExIpt;     // phase B tile: 4096 rids
constexpr uint64_t kExRange = 8ull * kExTile;         // phase A/B range: 32,768 rids
// Phase C and D items cover kExItemBytes of words: a grid of one 512-thread
// CTA per SM then works on about 152 x 256 KB = 39 MB of run order at a
// time, a few runs, which the L2 holds while they are probed.
constexpr uint64_t kExItemBytes = 256 * 1024;
// phase C items of the slot plan in the phase kernel (two CTAs per SM):
// 128 KB, so that the run order in flight (about 304 x 128 KB = 39 MB) stays
// inside the L2 with room for the INTERNAL lines being written
constexpr uint64_t kExItemBytesC = 128 * 1024;
// words a thread keeps in flight per round: UB bytes (128 in the fused
// kernel, 64 in the phase kernels that run two CTAs per SM), at most 16 words
template <int WB, int UB> __host__ __device__ constexpr int ex_u() { return UB / WB < 16 ? UB / WB : 16; }
constexpr int kExHistIpt = 32;                        // phase A: rids in flight per thread
constexpr uint32_t kExHistCopies = 8;                 // phase A: sub-histograms per CTA
constexpr uint32_t kExMaxRuns = 1024;
constexpr uint32_t kExListMax = 64;                   // requests a tile or chunk looks up in shared memory
constexpr uint32_t kExDone = 4;                       // done counters per group: A, B, C (and one spare)

enum : uint32_t { kPlanSlot = 0, kPlanScatter = 1 };
enum : uint32_t { kPhaseA = 0, kPhaseB = 1, kPhaseC = 2, kPhaseD = 3 };

struct ExReq {
  const uint8_t* rid_base;  // rid 0 of the request
  uint8_t* dst;             // its records (retrieval) or join rows
  const uint8_t* fact;      // join: the fact rows (rid i is the key of fact row i)
  uint64_t begin, n;        // the request's rids are group indices [begin, begin + n)
  uint32_t rid_stride;      // bytes between consecutive rids
  uint32_t n_src;           // each rid must be below this
};

struct ExGroup {
  const uint8_t* src;       // source records (the dimension table for a join)
  const uint8_t* rid_flat;  // rids in group order at a uniform stride, or null (then `rids`)
  uint32_t* cnt;            // G x nb: the place of range q inside run b
  uint32_t* tot;            // nb run totals (zeroed before the launch)
  int32_t* rids;            // group-order copy of the rids (phase A), when rid_flat is null
  uint32_t* run_rid;        // n rids in run order
  uint32_t* slot;           // slot plan: INTERNAL position of group rid t
  uint64_t* dptr;           // scatter plan: destination address of run position k
  uint8_t* internal;        // slot plan: n records in run order
  uint64_t n;               // rids in the group
  FastDiv fdW, fd_row;
  uint32_t rec, wb, W, sl, nb, G, req0, nreq, plan, join, fact_w, row_w, pk_off, rid_stride;
  uint64_t nC, nD;          // items of phases C and D
  uint64_t cwC, cwD;        // words of a phase C / phase D item
};

struct ExSeg {
  uint64_t first, count;    // items [first, first + count) of the global item space
  uint32_t phase, group;
};

// The request of group index t among reqs[a, a + m): the last with begin <= t.
__device__ __forceinline__ uint32_t ex_req_of(const ExReq* reqs, uint32_t a, uint32_t m, uint64_t t) {
  uint32_t lo = a, hi = a + m - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (reqs[mid].begin <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Exclusive scan of v[0, nb) into out[0, nb) by the whole block (nb <= 2 *
// kExThreads); wsum holds 32 words.
__device__ __forceinline__ void ex_scan(const uint32_t* v, uint32_t* out, uint32_t nb, uint32_t* wsum) {
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
    const uint32_t w = lane < (uint32_t)kExWarps ? wsum[lane] : 0u;
    uint32_t z = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= (uint32_t)o) z += y;
    }
    if (lane < (uint32_t)kExWarps) wsum[lane] = z - w;
  }
  __syncthreads();
  const uint32_t e = wsum[warp] + s - v0 - v1;
  if (x0 < nb) out[x0] = e;
  if (x0 + 1 < nb) out[x0 + 1] = e + v0;
  __syncthreads();
}

__device__ __forceinline__ int32_t ex_rid(const ExReq& r, uint64_t i) {
  return __ldg(reinterpret_cast<const int32_t*>(r.rid_base + i * r.rid_stride));
}

// Phase A, range q of group g.  h: kExHistCopies x nb words of shared
// memory: warp w counts into copy w % kExHistCopies, so that fewer threads
// meet on one counter (a few dozen runs take every rid).
__device__ __forceinline__ void ex_phase_a(const ExGroup& gs, const ExReq* __restrict__ reqs, uint64_t q,
                                           uint32_t* hs, int* err) {
  const ExGroup g = gs;  // fields in registers: the stores below cannot alias them
  for (uint32_t b = threadIdx.x; b < kExHistCopies * g.nb; b += kExThreads) hs[b] = 0;
  __syncthreads();
  uint32_t* h = hs + (threadIdx.x / 32 % kExHistCopies) * g.nb;
  const uint64_t lo = q * kExRange, hi = min(g.n, lo + kExRange);
  bool bad = false;
  for (uint32_t k = ex_req_of(reqs, g.req0, g.nreq, lo); k < g.req0 + g.nreq && reqs[k].begin < hi; ++k) {
    const ExReq r = reqs[k];
    const uint64_t a = max(lo, r.begin), z = min(hi, r.begin + r.n);
    for (uint64_t t0 = a + threadIdx.x; t0 < z; t0 += (uint64_t)kExHistIpt * kExThreads) {
      int32_t x[kExHistIpt];
#pragma unroll
      for (int u = 0; u < kExHistIpt; ++u) {
        const uint64_t t = t0 + (uint64_t)u * kExThreads;
        x[u] = t < z ? ex_rid(r, t - r.begin) : 0;
      }
#pragma unroll
      for (int u = 0; u < kExHistIpt; ++u) {
        const uint64_t t = t0 + (uint64_t)u * kExThreads;
        if (t < z) {
          if ((uint32_t)x[u] >= r.n_src) bad = true;
          else atomicAdd(&h[(uint32_t)x[u] >> g.sl], 1u);
          if (g.rids) g.rids[t] = x[u];
        }
      }
    }
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < g.nb; b += kExThreads) {
    uint32_t c = 0;
#pragma unroll
    for (uint32_t k = 0; k < kExHistCopies; ++k) c += hs[k * g.nb + b];
    g.cnt[q * g.nb + b] = c ? atomicAdd(&g.tot[b], c) : 0u;
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

// Shared memory of phase B: cur, tcnt, toff, delta, runoff (nb words each),
// the sorted tile's rids (kExTile words) and tile indices (kExTile halves),
// the tile's request list.
struct ExTileReqs {
  uint64_t begin[kExListMax];
  uint8_t* dst[kExListMax];
  uint32_t count;           // requests listed; kExListMax + 1: too many, search the table
  uint32_t first;
};

// Requests overlapping group indices [lo, hi) into L (thread 0 fills, all wait).
__device__ __forceinline__ void ex_list_reqs(uint32_t req0, uint32_t nreq, const ExReq* reqs, uint64_t lo,
                                             uint64_t hi, ExTileReqs& L) {
  if (threadIdx.x == 0) {
    const uint32_t k0 = ex_req_of(reqs, req0, nreq, lo);
    uint32_t m = 0;
    for (uint32_t k = k0; k < req0 + nreq && reqs[k].begin < hi; ++k, ++m) {
      if (m == kExListMax) {
        m = kExListMax + 1;
        break;
      }
      L.begin[m] = reqs[k].begin;
      L.dst[m] = reqs[k].dst;
    }
    L.count = m;
    L.first = k0;
  }
  __syncthreads();
}

// Request index (into L when listed, else the global table) and its begin /
// dst for group index t.
__device__ __forceinline__ void ex_lookup(uint32_t req0, uint32_t nreq, const ExReq* reqs, const ExTileReqs& L,
                                          uint64_t t, uint64_t& begin, uint8_t*& dst) {
  if (L.count <= kExListMax) {
    uint32_t lo = 0, hi = L.count - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (L.begin[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    begin = L.begin[lo];
    dst = L.dst[lo];
  } else {
    const uint32_t k = ex_req_of(reqs, req0, nreq, t);
    begin = reqs[k].begin;
    dst = reqs[k].dst;
  }
}

// Phase B, range q of group g.
__device__ __forceinline__ void ex_phase_b(const ExGroup& gs, const ExReq* __restrict__ reqs, uint64_t q,
                                           uint8_t* sm, uint32_t* wsum, ExTileReqs& L) {
  const ExGroup g = gs;
  const uint32_t nb = g.nb, tid = threadIdx.x;
  uint32_t* cur = reinterpret_cast<uint32_t*>(sm);
  uint32_t* tcnt = cur + nb;
  uint32_t* toff = tcnt + nb;
  uint32_t* delta = toff + nb;
  uint32_t* runoff = delta + nb;
  uint32_t* ent = runoff + nb;
  uint16_t* entt = reinterpret_cast<uint16_t*>(ent + kExTile);
  for (uint32_t x = tid; x < nb; x += kExThreads) tcnt[x] = __ldcg(g.tot + x);
  __syncthreads();
  ex_scan(tcnt, runoff, nb, wsum);
  for (uint32_t x = tid; x < nb; x += kExThreads) {
    cur[x] = runoff[x] + __ldcg(g.cnt + q * nb + x);
    tcnt[x] = 0;
  }
  __syncthreads();
  const uint64_t lo = q * kExRange, hi = min(g.n, lo + kExRange);
  const bool scatter = g.plan == kPlanScatter;
  // rids of tile t0 (group indices t0 + j), the next tile's loaded during this one
  auto load_tile = [&](uint64_t t0, uint32_t (&r)[kExIpt]) {
#pragma unroll
    for (int k = 0; k < kExIpt; ++k) {
      const uint64_t t = t0 + (uint64_t)k * kExThreads + tid;
      r[k] = 0;
      if (t < hi)
        r[k] = g.rid_flat ? (uint32_t)__ldg(reinterpret_cast<const int32_t*>(g.rid_flat + t * g.rid_stride))
                          : (uint32_t)__ldcg(g.rids + t);
    }
  };
  uint32_t r[kExIpt];
  load_tile(lo, r);
  for (uint64_t t0 = lo; t0 < hi; t0 += kExTile) {
    const uint32_t tn = (uint32_t)((hi - t0) < kExTile ? (hi - t0) : kExTile);
    uint32_t l[kExIpt], rn[kExIpt];
    load_tile(t0 + kExTile, rn);
    if (scatter) ex_list_reqs(g.req0, g.nreq, reqs, t0, t0 + tn, L);
#pragma unroll
    for (int k = 0; k < kExIpt; ++k)
      if (k * kExThreads + tid < tn) l[k] = atomicAdd(&tcnt[r[k] >> g.sl], 1u);
    __syncthreads();
    ex_scan(tcnt, toff, nb, wsum);
    for (uint32_t x = tid; x < nb; x += kExThreads) {
      delta[x] = cur[x] - toff[x];
      cur[x] += tcnt[x];
      tcnt[x] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kExIpt; ++k) {
      const uint32_t j = k * kExThreads + tid;
      if (j < tn) {
        const uint32_t b = r[k] >> g.sl;
        const uint32_t p = toff[b] + l[k];
        ent[p] = r[k];
        if (scatter) entt[p] = (uint16_t)j;
        else g.slot[t0 + j] = delta[b] + p;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kExIpt; ++k) {
      const uint32_t p = k * kExThreads + tid;
      if (p < tn) {
        const uint32_t rv = ent[p];
        const uint32_t pos = delta[rv >> g.sl] + p;
        g.run_rid[pos] = rv;
        if (scatter) {
          const uint64_t t = t0 + entt[p];
          uint64_t begin;
          uint8_t* dst;
          ex_lookup(g.req0, g.nreq, reqs, L, t, begin, dst);
          g.dptr[pos] = reinterpret_cast<uint64_t>(dst + (t - begin) * g.rec);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kExIpt; ++k) r[k] = rn[k];
  }
}

// Word t of a group's stream is word w of record k = t / W.  A thread's words
// in one round are t0 + u * kExThreads, u = 0, 1, ...: one division gives
// (k, w) for t0, and each next word adds kExThreads = q * W + rm, a 32-bit
// step (record indices fit 32 bits: a group holds fewer than 2^31 rids).
struct ExStep {
  uint32_t q, rm, W;
  __device__ __forceinline__ void next(uint32_t& k, uint32_t& w) const {
    k += q;
    w += rm;
    if (w >= W) {
      w -= W;
      ++k;
    }
  }
};

__device__ __forceinline__ ExStep ex_step(uint32_t W) {
  return ExStep{(uint32_t)kExThreads / W, (uint32_t)kExThreads % W, W};
}

// Phase C, item c of group g: words [c * cw, (c + 1) * cw) of the
// run-ordered record stream (cw = g.cwC).  Word t is word w of run
// position k, read from source record run_rid[k]; it goes to INTERNAL word t
// (slot plan) or to word w of run position k's destination record (scatter
// plan).  A join checks the key words of each dimension row (its int64 key
// at pk_off must equal the row number).  Each thread keeps U words in flight
// per round (the scatter plan also keeps their destination addresses, so at
// most 8) and loads the next round's rids while this round's records are on
// their way.
template <int WB, bool SCATTER, int UB>
__device__ __forceinline__ void ex_phase_c(const ExGroup& g, uint64_t c, int* err) {
  using T = typename WordT<WB>::T;
  // the fields used below, in registers (stores cannot alias them)
  const uint32_t* __restrict__ run_rid = g.run_rid;
  const uint64_t* __restrict__ dptr = g.dptr;
  const FastDiv fdW = g.fdW;
  const bool join = g.join != 0;
  const uint32_t pk_off = g.pk_off;
  constexpr int U = SCATTER ? (ex_u<WB, UB>() < 8 ? ex_u<WB, UB>() : 8) : ex_u<WB, UB>();
  const T* __restrict__ s = reinterpret_cast<const T*>(g.src);
  T* const iw0 = reinterpret_cast<T*>(g.internal);
  const uint32_t W = g.W;
  const ExStep st = ex_step(W);
  const uint64_t cw = g.cwC, i0 = c * cw, i1 = min(g.n * W, i0 + cw);
  const uint64_t step = (uint64_t)U * kExThreads;
  const uint32_t pk_w0 = pk_off / WB, pk_w1 = (pk_off + 8 + WB - 1) / WB;
  bool bad = false;
  // valid words of the round at r0, and the rids of its words
  auto count = [&](uint64_t r0) -> int {
    if (r0 >= i1) return 0;
    const uint64_t left = (i1 - r0 + kExThreads - 1) / kExThreads;
    return left < (uint64_t)U ? (int)left : U;
  };
  uint32_t id[U];
  auto load_ids = [&](uint64_t r0) {
    const int m = count(r0);
    uint32_t k = m ? (uint32_t)fdiv(r0, fdW) : 0u, w = m ? (uint32_t)(r0 - (uint64_t)k * W) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      id[u] = u < m ? run_rid[k] : 0u;
      st.next(k, w);
    }
  };
  load_ids(i0 + threadIdx.x);
  for (uint64_t r0 = i0 + threadIdx.x; r0 < i1; r0 += step) {
    const int m = count(r0);
    const uint32_t k0 = (uint32_t)fdiv(r0, fdW), w0 = (uint32_t)(r0 - (uint64_t)k0 * W);
    T v[U];
    T* to[SCATTER ? U : 1];
    {
      uint32_t k = k0, w = w0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < m) {
          v[u] = s[(uint64_t)id[u] * W + w];
          if constexpr (SCATTER) to[u] = reinterpret_cast<T*>(dptr[k]) + w;
        }
        st.next(k, w);
      }
    }
    if (join) {
      uint32_t k = k0, w = w0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < m && w >= pk_w0 && w < pk_w1 && !pk_word_ok<WB>(v[u], w, pk_off, id[u])) bad = true;
        st.next(k, w);
      }
    }
    load_ids(r0 + step);
    T* iw = iw0 + r0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < m) {
        if constexpr (SCATTER) *to[u] = v[u];
        else iw[u * kExThreads] = v[u];
      }
    }
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

// Phase D (slot plan), item c of group g: words [c * cw, (c + 1) * cw) of
// the group's destination stream in group order.  Retrieval: word w of group
// rid i is word w of INTERNAL record slot[i], stored in i's request (found in
// the item's request list; one request: no search).  Join (one request): row
// i is fact row i (fact_w words) then INTERNAL record slot[i] (W words).  The
// next round's slots are loaded while this round's words are on their way.
template <int WB, bool JOIN, int UB>
__device__ __forceinline__ void ex_phase_d(const ExGroup& g, const ExReq* __restrict__ reqs, uint64_t c,
                                           ExTileReqs& L) {
  using T = typename WordT<WB>::T;
  const uint32_t* __restrict__ slot = g.slot;
  constexpr int U = ex_u<WB, UB>();
  const T* __restrict__ iw = reinterpret_cast<const T*>(g.internal);
  const uint32_t W = g.W;
  const uint32_t row_w = JOIN ? g.row_w : W;
  const FastDiv fr = JOIN ? g.fd_row : g.fdW;
  const ExStep st = ex_step(row_w);
  const uint64_t cw = g.cwD, i0 = c * cw, i1 = min(g.n * row_w, i0 + cw);
  const uint64_t step = (uint64_t)U * kExThreads;
  auto count = [&](uint64_t r0) -> int {
    if (r0 >= i1) return 0;
    const uint64_t left = (i1 - r0 + kExThreads - 1) / kExThreads;
    return left < (uint64_t)U ? (int)left : U;
  };
  uint32_t sl[U];
  auto load_slots = [&](uint64_t r0) {
    const int m = count(r0);
    uint32_t i = m ? (uint32_t)fdiv(r0, fr) : 0u, w = m ? (uint32_t)(r0 - (uint64_t)i * row_w) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      sl[u] = u < m ? slot[i] : 0u;
      st.next(i, w);
    }
  };
  const uint8_t* fact = JOIN ? reqs[g.req0].fact : nullptr;
  uint8_t* out1 = JOIN ? reqs[g.req0].dst : nullptr;
  bool one = true;
  uint8_t* dst1 = out1;
  uint64_t begin1 = 0;
  if constexpr (!JOIN) {
    ex_list_reqs(g.req0, g.nreq, reqs, fdiv(i0, fr), fdiv(i1 - 1, fr) + 1, L);
    one = L.count == 1;
    dst1 = L.dst[0];
    begin1 = L.begin[0];
  }
  const T* fw = reinterpret_cast<const T*>(fact);
  const uint32_t fw_n = g.fact_w, req0 = g.req0, nreq = g.nreq;
  load_slots(i0 + threadIdx.x);
  for (uint64_t r0 = i0 + threadIdx.x; r0 < i1; r0 += step) {
    const int m = count(r0);
    const uint32_t i0r = (uint32_t)fdiv(r0, fr), w0r = (uint32_t)(r0 - (uint64_t)i0r * row_w);
    T v[U];
    {
      uint32_t i = i0r, w = w0r;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < m) {
          if (JOIN && w < fw_n) v[u] = __ldg(fw + (uint64_t)i * fw_n + w);
          else v[u] = iw[(uint64_t)sl[u] * W + (w - (JOIN ? fw_n : 0u))];
        }
        st.next(i, w);
      }
    }
    load_slots(r0 + step);
    if (JOIN || one) {
      T* o = reinterpret_cast<T*>(dst1) + (r0 - begin1 * row_w);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (u < m) o[u * kExThreads] = v[u];
    } else {
      uint32_t i = i0r, w = w0r;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < m) {
          uint64_t begin;
          uint8_t* dst;
          ex_lookup(req0, nreq, reqs, L, i, begin, dst);
          reinterpret_cast<T*>(dst)[(i - begin) * W + w] = v[u];
        }
        st.next(i, w);
      }
    }
  }
}

// Phases C and D for 4- and 8-byte words (records whose size is not a
// multiple of 16) written as 16-byte stores: chunk q is words [qV, qV + V) of
// the stream (V = 16 / WB), within one record or across two (W >= V); it is
// read as V words and stored as one 16-byte vector.  Phase C: the INTERNAL
// stream is 256-byte aligned.  Phase D: used for items that write one
// request (ex_phase_d16: the chunk grid follows the request's destination);
// items across requests take the word path.  Words past the last whole chunk
// of an item go word by word.
template <int WB>
__device__ __forceinline__ uint4 ex_pack(const typename WordT<WB>::T (&x)[16 / WB]) {
  if constexpr (WB == 4) return make_uint4(x[0], x[1], x[2], x[3]);
  else if constexpr (WB == 8) return make_uint4(x[0].x, x[0].y, x[1].x, x[1].y);
  else return x[0];
}

template <int WB, int UB>
__device__ __forceinline__ void ex_phase_c16(const ExGroup& g, uint64_t c, int* err) {
  using T = typename WordT<WB>::T;
  constexpr uint32_t V = 16 / WB;
  constexpr int UC = UB / 16;  // chunks in flight per thread
  const uint32_t* __restrict__ run_rid = g.run_rid;
  const T* __restrict__ s = reinterpret_cast<const T*>(g.src);
  uint4* const iv = reinterpret_cast<uint4*>(g.internal);
  T* const iw = reinterpret_cast<T*>(g.internal);
  const FastDiv fdW = g.fdW;
  const uint32_t W = g.W, pk_off = g.pk_off;
  const bool join = g.join != 0;
  const uint32_t pk_w0 = pk_off / WB, pk_w1 = (pk_off + 8 + WB - 1) / WB;
  const uint64_t cw = g.cwC, i0 = c * cw, i1 = min(g.n * W, i0 + cw);
  const uint64_t q0 = i0 / V, q1 = i1 / V;  // whole chunks [q0, q1); i0 is a multiple of V
  bool bad = false;
  auto word_ok = [&](const T& v, uint32_t w, uint32_t r) {
    return !join || w < pk_w0 || w >= pk_w1 || pk_word_ok<WB>(v, w, pk_off, r);
  };
  // the two source records of each chunk of a round (loaded a round ahead)
  uint32_t ra[UC], rb[UC], w0[UC];
  auto load_ids = [&](uint64_t qb) {
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      const uint64_t q = qb + (uint64_t)u * kExThreads;
      ra[u] = rb[u] = w0[u] = 0;
      if (q < q1) {
        const uint64_t t = q * V;
        const uint32_t k = (uint32_t)fdiv(t, fdW);
        w0[u] = (uint32_t)(t - (uint64_t)k * W);
        ra[u] = run_rid[k];
        rb[u] = w0[u] + V > W ? run_rid[k + 1] : ra[u];
      }
    }
  };
  load_ids(q0 + threadIdx.x);
  for (uint64_t qb = q0 + threadIdx.x; qb < q1; qb += (uint64_t)UC * kExThreads) {
    T x[UC][V];
    uint32_t ka[UC], kb[UC], ww[UC];
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      ka[u] = ra[u];
      kb[u] = rb[u];
      ww[u] = w0[u];
      if (qb + (uint64_t)u * kExThreads < q1) {
#pragma unroll
        for (uint32_t j = 0; j < V; ++j) {
          const uint32_t w = w0[u] + j;
          x[u][j] = w < W ? s[(uint64_t)ra[u] * W + w] : s[(uint64_t)rb[u] * W + (w - W)];
        }
      }
    }
    load_ids(qb + (uint64_t)UC * kExThreads);
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      const uint64_t q = qb + (uint64_t)u * kExThreads;
      if (q < q1) {
        if (join) {
#pragma unroll
          for (uint32_t j = 0; j < V; ++j) {
            const uint32_t w = ww[u] + j;
            if (!(w < W ? word_ok(x[u][j], w, ka[u]) : word_ok(x[u][j], w - W, kb[u]))) bad = true;
          }
        }
        iv[q] = ex_pack<WB>(x[u]);
      }
    }
  }
  // words after the last whole chunk (the stream's end)
  for (uint64_t t = q1 * V + threadIdx.x; t < i1; t += kExThreads) {
    const uint32_t k = (uint32_t)fdiv(t, fdW), w = (uint32_t)(t - (uint64_t)k * W);
    const uint32_t r = run_rid[k];
    const T v = s[(uint64_t)r * W + w];
    if (!word_ok(v, w, r)) bad = true;
    iw[t] = v;
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

// Phase D of a retrieval item writing one request as 16-byte chunks (see above).
// ex_phase_d16_range: stream words [i0, i1) of one request (begin, dst).
template <int WB, int UB>
__device__ __forceinline__ void ex_phase_d16_range(const ExGroup& g, uint64_t i0, uint64_t i1, uint8_t* dst,
                                                   uint64_t begin) {
  using T = typename WordT<WB>::T;
  constexpr uint32_t V = 16 / WB;
  constexpr int UC = UB / 16;
  const uint32_t* __restrict__ slot = g.slot;
  const T* __restrict__ iw = reinterpret_cast<const T*>(g.internal);
  const FastDiv fdW = g.fdW;
  const uint32_t W = g.W;
  const uint64_t b0 = begin * W;  // the request's first stream word; the words t >= b0
  const uint32_t sig = (uint32_t)(((reinterpret_cast<uintptr_t>(dst) / WB) % V + V - b0 % V) % V);
  const uint64_t q0 = (i0 + sig + V - 1) / V, q1 = (i1 + sig) / V;  // whole chunks [q0, q1)
  T* const dw = reinterpret_cast<T*>(dst);                        // dw[t - b0]: stream word t
  for (uint64_t qb = q0 + threadIdx.x; qb < q1; qb += (uint64_t)UC * kExThreads) {
    uint32_t sa[UC], sb[UC], w0[UC];
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      const uint64_t q = qb + (uint64_t)u * kExThreads;
      sa[u] = sb[u] = w0[u] = 0;
      if (q < q1) {
        const uint64_t t = q * V - sig;
        const uint32_t i = (uint32_t)fdiv(t, fdW);
        w0[u] = (uint32_t)(t - (uint64_t)i * W);
        sa[u] = slot[i];
        sb[u] = w0[u] + V > W ? slot[i + 1] : sa[u];
      }
    }
    T x[UC][V];
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      if (qb + (uint64_t)u * kExThreads < q1) {
#pragma unroll
        for (uint32_t j = 0; j < V; ++j) {
          const uint32_t w = w0[u] + j;
          x[u][j] = w < W ? iw[(uint64_t)sa[u] * W + w] : iw[(uint64_t)sb[u] * W + (w - W)];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      const uint64_t q = qb + (uint64_t)u * kExThreads;
      if (q < q1) *reinterpret_cast<uint4*>(dw + (q * V - sig - b0)) = ex_pack<WB>(x[u]);
    }
  }
  // words outside whole chunks: [i0, first chunk) and [after the last, i1)
  const uint64_t h1 = q1 > q0 ? q0 * V - sig : i1, t0 = q1 > q0 ? q1 * V - sig : i1;
  for (uint64_t t = i0 + threadIdx.x; t < h1; t += kExThreads) {
    const uint32_t i = (uint32_t)fdiv(t, fdW), w = (uint32_t)(t - (uint64_t)i * W);
    dw[t - b0] = iw[(uint64_t)slot[i] * W + w];
  }
  for (uint64_t t = t0 + threadIdx.x; t < i1; t += kExThreads) {
    const uint32_t i = (uint32_t)fdiv(t, fdW), w = (uint32_t)(t - (uint64_t)i * W);
    dw[t - b0] = iw[(uint64_t)slot[i] * W + w];
  }
}

template <int WB, int UB>
__device__ __forceinline__ void ex_phase_d16(const ExGroup& g, uint64_t c, uint8_t* dst, uint64_t begin) {
  const uint64_t i0 = c * g.cwD, i1 = min(g.n * g.W, i0 + g.cwD);
  ex_phase_d16_range<WB, UB>(g, i0, i1, dst, begin);
}

// Calls of the phase bodies go through these non-inlined wrappers where one
// kernel holds several of them (the fused kernel; the phase C and D kernels
// with their word sizes and plans), so that each is register-allocated on its
// own (inlined together they spill); the phase A and B kernels inline theirs.
__device__ __noinline__ void ex_call_a(const ExGroup& g, const ExReq* reqs, uint64_t q, uint32_t* h, int* err) {
  ex_phase_a(g, reqs, q, h, err);
}
__device__ __noinline__ void ex_call_b(const ExGroup& g, const ExReq* reqs, uint64_t q, uint8_t* sm, uint32_t* wsum,
                                       ExTileReqs& L) {
  ex_phase_b(g, reqs, q, sm, wsum, L);
}
template <int WB, bool SCATTER, int UB>
__device__ __noinline__ void ex_call_c(const ExGroup& g, uint64_t c, int* err) {
  ex_phase_c<WB, SCATTER, UB>(g, c, err);
}
template <int WB, bool JOIN, int UB>
__device__ __noinline__ void ex_call_d(const ExGroup& g, const ExReq* reqs, uint64_t c, ExTileReqs& L) {
  ex_phase_d<WB, JOIN, UB>(g, reqs, c, L);
}
template <int WB, int UB>
__device__ __noinline__ void ex_call_c16(const ExGroup& g, uint64_t c, int* err) {
  ex_phase_c16<WB, UB>(g, c, err);
}
template <int WB, int UB>
__device__ __noinline__ void ex_call_d16(const ExGroup& g, uint64_t c, uint8_t* dst, uint64_t begin) {
  ex_phase_d16<WB, UB>(g, c, dst, begin);
}

// Phase C or D of one item: 128 bytes in flight per thread in the fused
// kernel (one CTA per SM), 64 in the phase kernels (two CTAs per SM).
template <int WB, int PH>
__device__ __forceinline__ void ex_dispatch_cd(uint32_t phase, const ExGroup& g, const ExReq* reqs, uint64_t local,
                                               int* err, ExTileReqs& L) {
  constexpr int UB = PH < 0 ? 128 : 64;
  constexpr bool V16 = WB == 4 || WB == 8;  // 16-byte chunk stores available
  const bool chunks = V16 && g.W >= 16 / WB;
  if (phase == kPhaseC) {
    if (g.plan == kPlanScatter) ex_call_c<WB, true, UB>(g, local, err);
    else if constexpr (V16) {
      if (chunks) ex_call_c16<WB, UB>(g, local, err);
      else ex_call_c<WB, false, UB>(g, local, err);
    } else {
      ex_call_c<WB, false, UB>(g, local, err);
    }
  } else if (g.join) {
    ex_call_d<WB, true, UB>(g, reqs, local, L);
  } else {
    if constexpr (V16) {
      if (chunks) {
        // an item inside one request: the chunk path (at any WB-aligned destination)
        const uint64_t i0 = local * g.cwD, i1 = min(g.n * g.W, i0 + g.cwD);
        ex_list_reqs(g.req0, g.nreq, reqs, fdiv(i0, g.fdW), fdiv(i1 - 1, g.fdW) + 1, L);
        const uint64_t begin = L.begin[0];
        if (L.count == 1) {
          ex_call_d16<WB, UB>(g, local, L.dst[0], begin);
          return;
        }
      }
    }
    ex_call_d<WB, false, UB>(g, reqs, local, L);
  }
}

// The persistent executor.  done[] holds, per group, the finished items of
// phases B and C (at g * kExDone + phase) and, at done_a, the finished
// phase-A items of the whole batch.  Thread 0 claims the next item while the
// block works on the current one; an item never waits for an item claimed
// after it, and a claimed item is always the next one its CTA works on, so
// the smallest unfinished item can always run.
constexpr uint32_t kExSegCache = 128;  // segment table entries kept in shared memory

// PH < 0: the fused kernel, every phase of every item in one launch.
// PH >= 0: the kernel of one phase, items [item_base, n_items); its launch
// follows the previous phase's on the stream, so it waits for nothing.
template <int PH, int MINB>
__global__ void __launch_bounds__(kExThreads, MINB)
    k_exec(const ExGroup* __restrict__ groups, const ExReq* __restrict__ reqs, const ExSeg* __restrict__ segs,
           uint32_t nseg, uint64_t item_base, uint64_t n_items, uint32_t n_items_a, uint32_t* done,
           uint32_t* done_a, unsigned long long* ctr, int* err, long long wait_limit) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ uint32_t wsum[32];
  __shared__ ExTileReqs L;
  __shared__ ExSeg s_segs[kExSegCache];
  __shared__ __align__(16) ExGroup s_g;  // the current item's group (fields read from shared memory)
  __shared__ ExSeg s_sg;
  __shared__ uint64_t s_item, s_next;
  __shared__ uint32_t s_gidx, s_dep_group, s_dep_phase;
  __shared__ int s_go, s_copy;
  const bool cached = nseg <= kExSegCache;
  for (uint32_t x = threadIdx.x; cached && x < nseg; x += kExThreads) s_segs[x] = segs[x];
  if (threadIdx.x == 0) {
    s_gidx = s_dep_group = s_dep_phase = 0xffffffffu;
    s_next = error_set(err) ? n_items : item_base + atomicAdd(ctr, 1ull);
  }
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) {
      const uint64_t it = s_next;
      s_item = it;
      if (it < n_items) {
        // no new item once any error is set: a bad rid or a wait that ran out
        s_next = error_set(err) ? n_items : item_base + atomicAdd(ctr, 1ull);
        uint32_t lo = 0, hi = nseg - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if ((cached ? s_segs[mid].first : segs[mid].first) <= it) lo = mid;
          else hi = mid - 1;
        }
        s_sg = cached ? s_segs[lo] : segs[lo];
        s_copy = s_sg.group != s_gidx;
        s_gidx = s_sg.group;
      }
    }
    __syncthreads();
    const uint64_t it = s_item;
    if (it >= n_items) break;
    const ExSeg sg = s_sg;
    if (s_copy) {
      static_assert(sizeof(ExGroup) % 8 == 0, "the group descriptor is copied as 8-byte words");
      for (uint32_t x = threadIdx.x; x < sizeof(ExGroup) / 8; x += kExThreads)
        reinterpret_cast<uint64_t*>(&s_g)[x] = reinterpret_cast<const uint64_t*>(groups + sg.group)[x];
    }
    const ExGroup& g = s_g;
    const uint64_t local = it - sg.first;
    if (threadIdx.x == 0) {
      int go = 1;
      // wait for the earlier phase this item needs, unless this CTA has
      // already seen it complete (for phase B: every phase-A item of the batch)
      const uint32_t dg = sg.phase == kPhaseB ? 0xfffffffeu : sg.group;
      if (PH < 0 && sg.phase != kPhaseA && !(s_dep_group == dg && s_dep_phase == sg.phase)) {
        const uint32_t* word = sg.phase == kPhaseB ? done_a : done + (uint64_t)sg.group * kExDone + sg.phase - 1;
        const ExGroup& gg = groups[sg.group];
        const uint32_t need = sg.phase == kPhaseB ? n_items_a : sg.phase == kPhaseC ? gg.G : (uint32_t)gg.nC;
        bool ok;
        wait_word_bounded(word, wait_limit, &ok, [need, err](uint32_t x) { return x >= need || error_set(err); });
        if (!ok) atomicOr(err, ERR_TIMEOUT);
        __threadfence();
        if (ok && !error_set(err)) {
          s_dep_group = dg;
          s_dep_phase = sg.phase;
        }
      }
      // after a bad rid or a timeout nothing more is written
      if (sg.phase != kPhaseA && error_set(err)) go = 0;
      s_go = go;
    }
    __syncthreads();
    if (s_go) {
      if ((PH < 0 || PH == kPhaseA) && sg.phase == kPhaseA) {
        if constexpr (PH < 0) ex_call_a(g, reqs, local, reinterpret_cast<uint32_t*>(sm), err);
        else ex_phase_a(g, reqs, local, reinterpret_cast<uint32_t*>(sm), err);
      } else if ((PH < 0 || PH == kPhaseB) && sg.phase == kPhaseB) {
        if constexpr (PH < 0) ex_call_b(g, reqs, local, sm, wsum, L);
        else ex_phase_b(g, reqs, local, sm, wsum, L);
      } else if constexpr (PH < 0 || PH >= (int)kPhaseC) {
        switch (g.wb) {
          case 16: ex_dispatch_cd<16, PH>(sg.phase, g, reqs, local, err, L); break;
          case 8: ex_dispatch_cd<8, PH>(sg.phase, g, reqs, local, err, L); break;
          case 4: ex_dispatch_cd<4, PH>(sg.phase, g, reqs, local, err, L); break;
          case 2: ex_dispatch_cd<2, PH>(sg.phase, g, reqs, local, err, L); break;
          default: ex_dispatch_cd<1, PH>(sg.phase, g, reqs, local, err, L); break;
        }
      }
    }
    __syncthreads();
    if (PH < 0 && threadIdx.x == 0 && sg.phase != kPhaseD) {
      __threadfence();
      atomicAdd(sg.phase == kPhaseA ? done_a : done + (uint64_t)sg.group * kExDone + sg.phase, 1u);
    }
  }
}

// Phases C and D of the slot plan for groups of 4-, 8- or 16-byte words
// (WB = 4 from 3 words per record: a 16-byte chunk then spans at most two
// records), in kernels of their own: k_exec serves every word size, plan and join with
// one register allocation (64 registers, two CTAs per SM), where these run
// at the occupancy of the standalone gathers.  Items [item_base, n_items)
// are claimed in order as in k_exec.  Phase C (PH = kPhaseC, retrievals and
// joins): INTERNAL in run order as 16-byte chunks; SCATTER (the scatter
// plan's retrieval groups of 16-byte words): each record straight to its
// destination.  Phase D (retrievals): an
// item writes its stream words request by request, as 16-byte chunks
// aligned to each request's destination.
constexpr int kExD16MinBlocks = 4;
constexpr int kExD16Bytes = 32;  // bytes in flight per thread

template <int WB, int PH, bool SCATTER = false>
__global__ void __launch_bounds__(kExThreads, kExD16MinBlocks)
    k_exec_cd16(const ExGroup* __restrict__ groups, const ExReq* __restrict__ reqs, const ExSeg* __restrict__ segs,
                uint32_t nseg, uint64_t item_base, uint64_t n_items, unsigned long long* ctr, int* err) {
  __shared__ __align__(16) ExGroup s_g;
  __shared__ ExSeg s_sg;
  __shared__ uint64_t s_item, s_next;
  __shared__ uint32_t s_gidx, s_k0;
  __shared__ int s_copy, s_go;
  if (threadIdx.x == 0) {
    s_gidx = 0xffffffffu;
    s_next = error_set(err) ? n_items : item_base + atomicAdd(ctr, 1ull);
  }
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) {
      const uint64_t it = s_next;
      s_item = it;
      if (it < n_items) {
        // no new item once any error is set (a bad rid: nothing more is written)
        s_next = error_set(err) ? n_items : item_base + atomicAdd(ctr, 1ull);
        uint32_t lo = 0, hi = nseg - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (segs[mid].first <= it) lo = mid;
          else hi = mid - 1;
        }
        s_sg = segs[lo];
        s_copy = s_sg.group != s_gidx;
        s_gidx = s_sg.group;
        s_go = !error_set(err);
      }
    }
    __syncthreads();
    const uint64_t it = s_item;
    if (it >= n_items) break;
    if (s_copy)
      for (uint32_t x = threadIdx.x; x < sizeof(ExGroup) / 8; x += kExThreads)
        reinterpret_cast<uint64_t*>(&s_g)[x] = reinterpret_cast<const uint64_t*>(groups + s_sg.group)[x];
    __syncthreads();
    const ExGroup& g = s_g;
    if constexpr (PH == (int)kPhaseC) {
      if (s_go) {
        if constexpr (SCATTER) ex_phase_c<WB, true, kExD16Bytes>(g, it - s_sg.first, err);
        else ex_phase_c16<WB, kExD16Bytes>(g, it - s_sg.first, err);
      }
      __syncthreads();
      continue;
    }
    const uint64_t i0 = (it - s_sg.first) * g.cwD, i1 = min(g.n * g.W, i0 + g.cwD);
    if (threadIdx.x == 0) s_k0 = ex_req_of(reqs, g.req0, g.nreq, fdiv(i0, g.fdW));
    __syncthreads();
    if (s_go) {
      for (uint32_t k = s_k0; k < g.req0 + g.nreq; ++k) {
        const uint64_t b = reqs[k].begin;
        if (b * g.W >= i1) break;
        const uint64_t lo = max(i0, b * g.W), hi = min(i1, (b + reqs[k].n) * g.W);
        if (lo < hi) ex_phase_d16_range<WB, kExD16Bytes>(g, lo, hi, reqs[k].dst, b);
      }
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace dpg

// ------------------------------------------------------------------ host side

namespace dpg {
namespace {

size_t ex_al(size_t x) { return (x + 255) & ~size_t(255); }

// One live request of the batch, normalized.
struct ExLive {
  bool join;
  const uint8_t* src;   // source (dimension) table
  uint64_t n_src;
  uint32_t rec;         // source record (dimension row) bytes
  uint64_t n;           // rids (fact rows)
  const uint8_t* rid_base;
  uint32_t rid_stride;
  uint8_t* dst;
  const uint8_t* fact;  // join
  uint32_t fact_bytes, pk_off;
};

// Runs of about run_bytes of source, at most kExMaxRuns of them.
uint32_t ex_run_log2(uint64_t n_src, uint32_t rec, uint64_t run_bytes) {
  uint32_t k = 0;
  while (k < 31 && ((2ull << k) * rec) <= run_bytes) ++k;
  while (k < 31 && ((n_src + (1ull << k) - 1) >> k) > kExMaxRuns) ++k;
  return k;
}

bool ex_overlap(const void* a, uint64_t na, const void* b, uint64_t nb) {
  if (!na || !nb) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

// Host-side checks and normalization of one item (DPG_OK, DPG_EINVAL).
int ex_normalize(const dpg_batch_item& it, ExLive* out, bool* live) {
  const dpg_job& j = it.job;
  *live = false;
  if (j.kind == DPG_JOB_RETRIEVE) {
    if (j.rec_bytes == 0 || j.rec_bytes > kMaxDpgRecBytes || j.n > 0x7fffffffULL || j.n_src > 0x7fffffffULL)
      return DPG_EINVAL;
    if (j.n == 0) return DPG_OK;
    if (!j.rids || !it.out || (j.n_src && !j.src) || reinterpret_cast<uintptr_t>(j.rids) % 4) return DPG_EINVAL;
    if (ex_overlap(j.src, j.n_src * j.rec_bytes, it.out, j.n * j.rec_bytes) ||
        ex_overlap(j.rids, j.n * 4, it.out, j.n * j.rec_bytes))
      return DPG_EINVAL;
    *out = ExLive{false, static_cast<const uint8_t*>(j.src), j.n_src, (uint32_t)j.rec_bytes, j.n,
                  reinterpret_cast<const uint8_t*>(j.rids), 4u, static_cast<uint8_t*>(it.out), nullptr, 0u, 0u};
    *live = true;
    return DPG_OK;
  }
  if (j.kind == DPG_JOB_JOIN) {
    if (j.join_mode != DPG_JOIN_MOVE) return DPG_EINVAL;
    if (j.fact_bytes < 4 || j.fact_bytes % 4 || j.fk_off % 4 || j.fk_off + 4 > j.fact_bytes) return DPG_EINVAL;
    if (j.dim_bytes < 8 || j.pk_off + 8 > j.dim_bytes) return DPG_EINVAL;
    if (j.n_fact > 0x7fffffffULL || j.n_dim > 0x7fffffffULL || j.fact_bytes > kMaxDpgRecBytes ||
        j.dim_bytes > kMaxDpgRecBytes)
      return DPG_EINVAL;
    if (!fastdiv_exact((uint32_t)(j.fact_bytes + j.dim_bytes), (uint64_t)j.n_fact * (j.fact_bytes + j.dim_bytes)))
      return DPG_EINVAL;
    if (j.n_fact == 0) return DPG_OK;
    if (!j.fact || !it.out || (j.n_dim && !j.dim) || reinterpret_cast<uintptr_t>(j.fact) % 4) return DPG_EINVAL;
    const uint64_t out_bytes = j.n_fact * (j.fact_bytes + j.dim_bytes);
    if (ex_overlap(j.fact, j.n_fact * j.fact_bytes, it.out, out_bytes) ||
        ex_overlap(j.dim, j.n_dim * j.dim_bytes, it.out, out_bytes))
      return DPG_EINVAL;
    const uint8_t* fact = static_cast<const uint8_t*>(j.fact);
    *out = ExLive{true, static_cast<const uint8_t*>(j.dim), j.n_dim, (uint32_t)j.dim_bytes, j.n_fact,
                  fact + j.fk_off, (uint32_t)j.fact_bytes, static_cast<uint8_t*>(it.out), fact,
                  (uint32_t)j.fact_bytes, (uint32_t)j.pk_off};
    *live = true;
    return DPG_OK;
  }
  return DPG_EINVAL;
}

// Plan of a retrieval group: an environment override (DPG_EXEC_PLAN = slot or
// scatter), else the plan dpg_tune cached for the group's shape (the L2-run
// plan -> slot plan with its run length; a shared-memory plan -> scatter
// plan), else slot below 192-byte records and scatter from 192 bytes (where
// the fused 2-pass plan wins in the record-size sweep).
void ex_plan(const dpg_ctx& c, const ExLive& q0, uint64_t n_src, uint64_t n, uint32_t* plan, uint32_t* sl) {
  *plan = q0.rec < 192 ? kPlanSlot : kPlanScatter;
  *sl = ex_run_log2(n_src, q0.rec, (uint64_t)env_int("DPG_L2_RUN_KB", 16384) << 10);
  Retrieval r{q0.src, n_src, q0.rec, n, RidSpec{q0.rid_base, 4}, nullptr, nullptr};
  auto it = c.plans.find(plan_key(r));
  if (it != c.plans.end()) {
    // the tuner's 2-pass plan (Phase II writes each record at its
    // destination) is the scatter plan; its L2-run and 3-pass plans (Phase II
    // writes INTERNAL, Phase III gathers) are the slot plan, which also takes
    // the tuned run length of an L2-run plan
    *plan = it->second.first == 2 ? kPlanScatter : kPlanSlot;
    if (it->second.first == 4 && ((n_src + (1ull << it->second.second) - 1) >> it->second.second) <= kExMaxRuns)
      *sl = (uint32_t)it->second.second;
  }
  const char* e = std::getenv("DPG_EXEC_PLAN");
  if (e && !std::strcmp(e, "slot")) *plan = kPlanSlot;
  if (e && !std::strcmp(e, "scatter")) *plan = kPlanScatter;
}

}  // namespace

int run_exec_batch(dpg_ctx& c, const dpg_batch_item* items, size_t count, cudaStream_t st) {
  if (count && !items) return DPG_EINVAL;
  std::vector<ExLive> live;
  live.reserve(count);
  for (size_t k = 0; k < count; ++k) {
    ExLive q;
    bool is_live = false;
    if (int s = ex_normalize(items[k], &q, &is_live)) return s;
    if (is_live) live.push_back(q);
  }
  if (live.empty()) return DPG_OK;
  const bool fused = env_int("DPG_EXEC_FUSED", 0) != 0;
  // groups: retrievals of one source table and record size (in submission
  // order inside the group); every join alone
  std::vector<size_t> order(live.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    const ExLive &a = live[x], &b = live[y];
    if (a.join != b.join) return !a.join;
    if (a.join) return false;
    if (a.src != b.src) return reinterpret_cast<uintptr_t>(a.src) < reinterpret_cast<uintptr_t>(b.src);
    return a.rec < b.rec;
  });
  std::vector<ExGroup> groups;
  std::vector<ExReq> reqs;
  for (size_t i = 0; i < order.size();) {
    const ExLive& q0 = live[order[i]];
    size_t j = i + 1;
    if (!q0.join)
      while (j < order.size() && !live[order[j]].join && live[order[j]].src == q0.src && live[order[j]].rec == q0.rec)
        ++j;
    ExGroup g{};
    g.src = q0.src;
    g.rec = q0.rec;
    g.join = q0.join ? 1u : 0u;
    g.req0 = (uint32_t)reqs.size();
    g.nreq = (uint32_t)(j - i);
    uint64_t n_src = 0;
    bool flat = true;
    uint32_t wb = std::min(pow2_align(q0.rec), pow2_align(reinterpret_cast<uintptr_t>(q0.src)));
    for (size_t k = i; k < j; ++k) {
      const ExLive& q = live[order[k]];
      if (q.rid_stride != q0.rid_stride || q.rid_base != q0.rid_base + (uint64_t)q0.rid_stride * g.n) flat = false;
      reqs.push_back(ExReq{q.rid_base, q.dst, q.fact, g.n, q.n, q.rid_stride, (uint32_t)q.n_src});
      g.n += q.n;
      n_src = std::max(n_src, q.n_src);
      wb = std::min(wb, pow2_align(reinterpret_cast<uintptr_t>(q.dst)));
    }
    if (g.n > 0x7fffffffULL) return DPG_EINVAL;  // run positions and slots are 32-bit
    if (g.join) {
      wb = std::min({wb, pow2_align(q0.fact_bytes), pow2_align(reinterpret_cast<uintptr_t>(q0.fact))});
      g.plan = kPlanSlot;
      g.sl = ex_run_log2(n_src, q0.rec, (uint64_t)env_int("DPG_L2_RUN_KB", 16384) << 10);
      g.pk_off = q0.pk_off;
    } else {
      ex_plan(c, q0, n_src, g.n, &g.plan, &g.sl);
    }
    g.wb = wb;
    g.W = q0.rec / wb;
    g.fdW = make_fastdiv(g.W);
    g.fact_w = g.join ? q0.fact_bytes / wb : 0u;
    g.row_w = g.fact_w + g.W;
    g.fd_row = make_fastdiv(g.row_w);
    g.nb = std::max<uint32_t>(1, (uint32_t)((n_src + (1ull << g.sl) - 1) >> g.sl));
    g.G = (uint32_t)((g.n + kExRange - 1) / kExRange);
    g.cwC = (fused || g.plan == kPlanScatter ? kExItemBytes : kExItemBytesC) / wb;
    g.cwD = kExItemBytes / wb;
    g.nC = (g.n * g.W + g.cwC - 1) / g.cwC;
    g.nD = g.plan == kPlanSlot ? (g.n * (g.join ? g.row_w : g.W) + g.cwD - 1) / g.cwD : 0;
    g.rid_flat = flat ? q0.rid_base : nullptr;
    g.rid_stride = q0.rid_stride;
    groups.push_back(g);
    i = j;
  }
  // items, phase by phase; phase D in three runs: the retrieval groups of
  // 4-byte words and of 8-byte words (k_exec_d16), then the rest
  // items, phase by phase; phases C and D in runs: the groups k_exec_cd16
  // takes, by word size and plan (phase D: retrievals only), then the rest
  // run of a group's phase-C or phase-D items: 0, 1, 2 the lean kernel for
  // 4-, 8-, 16-byte words; 3 (phase C) the lean scatter kernel; 4 the rest
  auto cd_pass = [](const ExGroup& g, uint32_t ph) -> int {
    if (ph == kPhaseC && g.plan == kPlanScatter && g.wb == 16 && !g.join) return 3;
    const bool words = g.wb == 16 || g.wb == 8 || (g.wb == 4 && g.W >= 3);
    if (g.plan != kPlanSlot || !words || (ph == kPhaseD && g.join)) return 4;
    return g.wb == 4 ? 0 : g.wb == 8 ? 1 : 2;
  };
  std::vector<ExSeg> segs;
  uint64_t n_items = 0, n_a = 0;
  uint64_t cd_run[2][6] = {};  // phase C / D item boundaries by run (cd_pass), then the end
  for (uint32_t ph = kPhaseA; ph <= kPhaseD; ++ph) {
    const bool split = ph >= kPhaseC;
    for (int pass = 0; pass < (split ? 5 : 1); ++pass) {
      if (split) cd_run[ph - kPhaseC][pass] = n_items;
      for (uint32_t gi = 0; gi < groups.size(); ++gi) {
        const ExGroup& g = groups[gi];
        if (split && cd_pass(g, ph) != pass) continue;
        const uint64_t cntp = ph <= kPhaseB ? g.G : ph == kPhaseC ? g.nC : g.nD;
        if (!cntp) continue;
        segs.push_back(ExSeg{n_items, cntp, ph, gi});
        n_items += cntp;
        if (ph == kPhaseA) n_a += cntp;
      }
    }
    if (split) cd_run[ph - kPhaseC][5] = n_items;
  }
  if (n_a > 0xffffffffULL) return DPG_EINVAL;
  // work space: the zeroed header (phase-A counter, item counter, done
  // counters, run totals), the tables, then each group's buffers
  const size_t ng = groups.size();
  size_t at = 256 + ex_al(ng * kExDone * 4);
  std::vector<size_t> tot_at(ng);
  for (size_t gi = 0; gi < ng; ++gi) {
    tot_at[gi] = at;
    at += ex_al(groups[gi].nb * 4);
  }
  const size_t zero_bytes = at;
  const size_t tab_at = at;
  const size_t tab_bytes = ex_al(ng * sizeof(ExGroup)) + ex_al(reqs.size() * sizeof(ExReq)) +
                           ex_al(segs.size() * sizeof(ExSeg));
  at += tab_bytes;
  struct Bufs { size_t cnt, rids, run, side, internal; };
  std::vector<Bufs> bufs(ng);
  uint32_t nb_max = 1;
  for (size_t gi = 0; gi < ng; ++gi) {
    const ExGroup& g = groups[gi];
    nb_max = std::max(nb_max, g.nb);
    bufs[gi].cnt = at; at += ex_al((size_t)g.G * g.nb * 4);
    bufs[gi].rids = at; at += g.rid_flat ? 0 : ex_al(g.n * 4);
    bufs[gi].run = at; at += ex_al(g.n * 4);
    bufs[gi].side = at; at += ex_al(g.n * (g.plan == kPlanSlot ? 4 : 8));
    bufs[gi].internal = at; at += g.plan == kPlanSlot ? ex_al(g.n * g.rec) : 0;
  }
  if (int s = ensure_aux(c, at)) return s;
  uint8_t* base = static_cast<uint8_t*>(c.aux);
  for (size_t gi = 0; gi < ng; ++gi) {
    ExGroup& g = groups[gi];
    const Bufs& b = bufs[gi];
    g.tot = reinterpret_cast<uint32_t*>(base + tot_at[gi]);
    g.cnt = reinterpret_cast<uint32_t*>(base + b.cnt);
    g.rids = g.rid_flat ? nullptr : reinterpret_cast<int32_t*>(base + b.rids);
    g.run_rid = reinterpret_cast<uint32_t*>(base + b.run);
    g.slot = g.plan == kPlanSlot ? reinterpret_cast<uint32_t*>(base + b.side) : nullptr;
    g.dptr = g.plan == kPlanScatter ? reinterpret_cast<uint64_t*>(base + b.side) : nullptr;
    g.internal = g.plan == kPlanSlot ? base + b.internal : nullptr;
  }
  // tables staged in context-owned pinned memory (a replayed graph reads it again)
  if (c.batch_host_bytes < tab_bytes) {
    if (c.batch_host) cudaFreeHost(c.batch_host);
    c.batch_host = nullptr;
    c.batch_host_bytes = 0;
    if (cudaMallocHost(&c.batch_host, tab_bytes) != cudaSuccess) {
      cudaGetLastError();
      return DPG_ENOMEM;
    }
    c.batch_host_bytes = tab_bytes;
  }
  uint8_t* h = static_cast<uint8_t*>(c.batch_host);
  std::memcpy(h, groups.data(), ng * sizeof(ExGroup));
  std::memcpy(h + ex_al(ng * sizeof(ExGroup)), reqs.data(), reqs.size() * sizeof(ExReq));
  std::memcpy(h + ex_al(ng * sizeof(ExGroup)) + ex_al(reqs.size() * sizeof(ExReq)), segs.data(),
              segs.size() * sizeof(ExSeg));
  const ExGroup* d_groups = reinterpret_cast<const ExGroup*>(base + tab_at);
  const ExReq* d_reqs = reinterpret_cast<const ExReq*>(base + tab_at + ex_al(ng * sizeof(ExGroup)));
  const ExSeg* d_segs =
      reinterpret_cast<const ExSeg*>(base + tab_at + ex_al(ng * sizeof(ExGroup)) + ex_al(reqs.size() * sizeof(ExReq)));
  cudaError_t e = cudaMemsetAsync(base, 0, zero_bytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + tab_at, h, tab_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch tables");
  const size_t smem = std::max<size_t>(20 * (size_t)nb_max + kExTile * 6, (size_t)kExHistCopies * 4 * nb_max);
  uint32_t* d_done = reinterpret_cast<uint32_t*>(base + 256);
  uint32_t* d_done_a = reinterpret_cast<uint32_t*>(base);
  unsigned long long* d_ctr = reinterpret_cast<unsigned long long*>(base + 8);  // 12 counters
  if (fused) {
    // one launch: every phase, dependencies by bounded waits
    auto kern = k_exec<-1, 1>;
    set_smem(kern, smem);
    const int per_sm = resident_per_sm(kern, kExThreads, smem);
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(n_items, (uint64_t)c.sms * per_sm));
    TraceScope ts(c, "k_exec", st);
    kern<<<(uint32_t)grid, kExThreads, smem, st>>>(d_groups, d_reqs, d_segs, (uint32_t)segs.size(), 0, n_items,
                                                   (uint32_t)n_a, d_done, d_done_a, d_ctr, c.d_err, c.wait_cycles);
    c.launches++;
  } else {
    // one persistent launch per phase over that phase's items of every group
    uint64_t ph_begin[5] = {0, 0, 0, 0, 0};
    for (const ExSeg& sg : segs) ph_begin[sg.phase + 1] = sg.first + sg.count;
    for (int ph = 1; ph <= 4; ++ph) ph_begin[ph] = std::max(ph_begin[ph], ph_begin[ph - 1]);
    auto launch = [&](auto kern, int ph, size_t ph_smem, const char* name) {
      const uint64_t lo = ph_begin[ph], hi = ph_begin[ph + 1];
      if (hi <= lo) return;
      set_smem(kern, ph_smem);
      const int per_sm = resident_per_sm(kern, kExThreads, ph_smem);
      const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(hi - lo, (uint64_t)c.sms * per_sm));
      TraceScope ts(c, name, st);
      kern<<<(uint32_t)grid, kExThreads, ph_smem, st>>>(d_groups, d_reqs, d_segs, (uint32_t)segs.size(), lo, hi,
                                                        (uint32_t)n_a, d_done, d_done_a, d_ctr + 1 + ph, c.d_err,
                                                        c.wait_cycles);
      c.launches++;
    };
    // phases A and B: three CTAs per SM (40 registers); C and D: two (64)
    launch(k_exec<kPhaseA, 3>, kPhaseA, (size_t)kExHistCopies * 4 * nb_max, "k_exec_a");
    launch(k_exec<kPhaseB, 3>, kPhaseB, 20 * (size_t)nb_max + kExTile * 6, "k_exec_b");
    // phases C and D: three runs of items each, each run with a counter of its own
    auto launch_cd16 = [&](auto kern, uint64_t lo, uint64_t hi, unsigned long long* ctr, const char* name) {
      if (hi <= lo) return;
      const int per_sm = resident_per_sm(kern, kExThreads, 0);
      const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(hi - lo, (uint64_t)c.sms * per_sm));
      TraceScope ts(c, name, st);
      kern<<<(uint32_t)grid, kExThreads, 0, st>>>(d_groups, d_reqs, d_segs, (uint32_t)segs.size(), lo, hi, ctr,
                                                  c.d_err);
      c.launches++;
    };
    const uint64_t(&cr)[6] = cd_run[0];
    const uint64_t(&dr)[6] = cd_run[1];
    launch_cd16(k_exec_cd16<4, kPhaseC>, cr[0], cr[1], d_ctr + 5, "k_exec_c16");
    launch_cd16(k_exec_cd16<8, kPhaseC>, cr[1], cr[2], d_ctr + 6, "k_exec_c16");
    launch_cd16(k_exec_cd16<16, kPhaseC>, cr[2], cr[3], d_ctr + 7, "k_exec_c16");
    launch_cd16(k_exec_cd16<16, kPhaseC, true>, cr[3], cr[4], d_ctr + 11, "k_exec_cs16");
    ph_begin[kPhaseC] = cr[4];  // the rest of phase C
    launch(k_exec<kPhaseC, 2>, kPhaseC, 0, "k_exec_c");
    launch_cd16(k_exec_cd16<4, kPhaseD>, dr[0], dr[1], d_ctr + 8, "k_exec_d16");
    launch_cd16(k_exec_cd16<8, kPhaseD>, dr[1], dr[2], d_ctr + 9, "k_exec_d16");
    launch_cd16(k_exec_cd16<16, kPhaseD>, dr[2], dr[3], d_ctr + 10, "k_exec_d16");
    ph_begin[kPhaseD] = dr[4];  // the rest of phase D
    launch(k_exec<kPhaseD, 2>, kPhaseD, 0, "k_exec_d");
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? DPG_OK : cuda_fail(c, e, "batch executor launch");
}

}  // namespace dpg

extern "C" dpg_status dpg_run_batch(dpg_ctx* c, const dpg_batch_item* items, size_t count, void* stream) {
  if (!c) return DPG_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  const int s = dpg::run_exec_batch(*c, items, count, static_cast<cudaStream_t>(stream));
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return (dpg_status)s;
}
