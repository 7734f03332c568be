// Record retrieval kernels for sm_103a: distribute-probe-gather (DPG, §2.1 and
// Figure 1 of Cooperman, Ma, Nguyen) and the plain one-pass gather (§1).
//
// Notation: N = n_src source records of `rec` bytes, n rids, segments (the
// paper's runs) of S = 2^seg_log2 consecutive source records, nb = ceil(N/S)
// segments.  All arithmetic is integer.
//
//   K2 k_hist        Phase I, pass 1: per-CTA counts of rids per segment,
//                    range check of every rid (before any destination write).
//   K3 k_scan        Phase I: run offsets (exclusive scan of the counts),
//                    per-(segment, CTA) write cursors and probe work items
//                    (a segment with many rids is split into chunks, §2.3).
//   K4 k_distribute  Phase I, pass 2: append each rid's in-segment offset to
//                    its run (RID_RUN) and remember where it went.
//   K5 k_probe       Phase II: bulk-copy one source segment into shared memory
//                    (cp.async.bulk + mbarrier), then copy its records out in
//                    run order, into the INTERNAL staging table (3-pass plan)
//                    or straight into their destination slots (2-pass plan).
//   K6 k_gather      Phase III: dst[i] = INTERNAL[slot[i]], written in rid
//                    order as one coalesced stream (k_gather16 when records
//                    are a multiple of 4 or 8 bytes but not of 16).
//   K1 k_gather      the baseline: dst[i] = src[rids[i]] in one pass.
//
// These are the plans with shared-memory segments (3-pass and 2-pass); the
// plan with runs held in the L2 is in dpg_runs.cu.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>

#include "dpg_device.cuh"
#include "dpg_internal.h"
#include "dpg_launch.cuh"
#include "dpg_scan.cuh"

namespace dpg {
namespace {

constexpr int kGatherThreads = 256;
constexpr int kGatherUnroll = 8;
constexpr int kPhaseThreads = 1024;
constexpr int kProbeThreads = 512;
constexpr uint32_t kSegBytesMax = 104 * 1024;  // two probe CTAs per SM (segment + staged run entries)
constexpr uint32_t kBulkPiece = 32 * 1024;     // bytes per cp.async.bulk request
constexpr int kHistUnroll = 8;

// --------------------------------------------------------------- K1 / K6
// dst[i] = src[idx(i)] for i in [0, n).  The destination is one contiguous
// stream of WB-byte words; word t belongs to record i = t / W, word w = t % W,
// and is read from word w of source record idx(i).  Each thread keeps
// kGatherUnroll independent loads in flight.
template <int WB, bool CHECK, class Idx>
__global__ void __launch_bounds__(kGatherThreads)
    k_gather(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, Idx idx, uint64_t n, uint32_t W,
             FastDiv fdW, uint32_t n_src, int* err) {
  using T = typename WordT<WB>::T;
  if (!CHECK && error_set(err)) return;
  const T* s = reinterpret_cast<const T*>(src);
  T* d = reinterpret_cast<T*>(dst);
  const uint64_t total = n * W;
  const uint64_t step = (uint64_t)gridDim.x * kGatherThreads * kGatherUnroll;
  bool bad = false;
  for (uint64_t base = (uint64_t)blockIdx.x * kGatherThreads * kGatherUnroll + threadIdx.x; base < total;
       base += step) {
    T v[kGatherUnroll];
    bool ok[kGatherUnroll];
#pragma unroll
    for (int k = 0; k < kGatherUnroll; ++k) {
      const uint64_t t = base + (uint64_t)k * kGatherThreads;
      ok[k] = false;
      if (t < total) {
        const uint64_t i = fdiv(t, fdW);
        const uint32_t w = (uint32_t)(t - i * W);
        const uint32_t r = (uint32_t)idx(i);
        if (!CHECK || r < n_src) {
          v[k] = s[(uint64_t)r * W + w];
          ok[k] = true;
        } else {
          bad = true;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kGatherUnroll; ++k)
      if (ok[k]) d[base + (uint64_t)k * kGatherThreads] = v[k];
  }
  if (CHECK && bad) atomicOr(err, ERR_RANGE);
}

// The same gather with the destination written as 16-byte vectors, for
// WB = 4 or 8 (records whose size is not a multiple of 16), W >= V = 16 / WB
// and a 16-byte-aligned destination.  Chunk c is words [V*c, V*c + V) of the
// destination word stream; it spans at most two records and is assembled
// from V WB-byte loads.  Two chunks per thread keep 32 bytes in flight, which
// measured best on the Phase III slot pattern (fewer store instructions and
// divisions than one word per thread).  The last total % V words are written
// one by one by block 0.  With CHECK, a chunk that touches a rid outside
// [0, n_src) writes only its words from valid records.
constexpr int kGather16Unroll = 2;

template <int WB, bool CHECK, class Idx>
__global__ void __launch_bounds__(kGatherThreads)
    k_gather16(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, Idx idx, uint64_t n, uint32_t W,
               FastDiv fdW, uint32_t n_src, int* err) {
  static_assert(WB == 4 || WB == 8, "16-byte chunks of 4- or 8-byte words");
  using T = typename WordT<WB>::T;
  constexpr uint32_t V = 16 / WB;
  if (!CHECK && error_set(err)) return;
  const T* s = reinterpret_cast<const T*>(src);
  T* dw = reinterpret_cast<T*>(dst);
  uint4* d = reinterpret_cast<uint4*>(dst);
  const uint64_t total = n * W, C = total / V;
  const uint64_t step = (uint64_t)gridDim.x * kGatherThreads * kGather16Unroll;
  bool bad = false;
  for (uint64_t base = (uint64_t)blockIdx.x * kGatherThreads * kGather16Unroll + threadIdx.x; base < C;
       base += step) {
    T x[kGather16Unroll][V];
    bool ok[kGather16Unroll];
#pragma unroll
    for (int k = 0; k < kGather16Unroll; ++k) {
      const uint64_t c = base + (uint64_t)k * kGatherThreads;
      ok[k] = c < C;
      if (!ok[k]) continue;
      const uint64_t t0 = (uint64_t)V * c;
      const uint64_t i0 = fdiv(t0, fdW);
      const uint32_t w0 = (uint32_t)(t0 - i0 * W);
      const uint32_t r0 = (uint32_t)idx(i0);
      const uint32_t r1 = (w0 + V > W) ? (uint32_t)idx(i0 + 1) : r0;
      if (CHECK && (r0 >= n_src || r1 >= n_src)) {
        bad = true;
        ok[k] = false;
#pragma unroll
        for (uint32_t j = 0; j < V; ++j) {
          const uint32_t w = w0 + j;
          const uint32_t r = w < W ? r0 : r1;
          if (r < n_src) dw[t0 + j] = s[(uint64_t)r * W + (w < W ? w : w - W)];
        }
        continue;
      }
#pragma unroll
      for (uint32_t j = 0; j < V; ++j) {
        const uint32_t w = w0 + j;
        x[k][j] = w < W ? s[(uint64_t)r0 * W + w] : s[(uint64_t)r1 * W + (w - W)];
      }
    }
#pragma unroll
    for (int k = 0; k < kGather16Unroll; ++k) {
      if (!ok[k]) continue;
      uint4 v;
      if constexpr (WB == 4) v = make_uint4(x[k][0], x[k][1], x[k][2], x[k][3]);
      else v = make_uint4(x[k][0].x, x[k][0].y, x[k][1].x, x[k][1].y);
      d[base + (uint64_t)k * kGatherThreads] = v;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < total - C * V) {
    const uint64_t t = C * V + threadIdx.x;
    const uint64_t i = fdiv(t, fdW);
    const uint32_t w = (uint32_t)(t - i * W);
    const uint32_t r = (uint32_t)idx(i);
    if (!CHECK || r < n_src) dw[t] = s[(uint64_t)r * W + w];
    else bad = true;
  }
  if (CHECK && bad) atomicOr(err, ERR_RANGE);
}

// --------------------------------------------------------------------- K2
// CTA g counts the rids of [g*per, (g+1)*per) per segment in shared memory and
// writes them as row g of the CTA-major count matrix cnt[g*nb + b].  With more
// segments than shared counters (smem_mode == 0) it counts straight into the
// segment totals tot[] with global atomics.
template <class Rid>
__global__ void __launch_bounds__(kPhaseThreads)
    k_hist(Rid rid, uint64_t n, uint32_t n_src, uint32_t seg_log2, uint32_t nb, uint32_t G, uint64_t per,
           uint32_t* __restrict__ cnt, uint32_t* __restrict__ tot, int* err, int smem_mode,
           int32_t* __restrict__ compact) {
  extern __shared__ uint32_t h[];
  const uint32_t g = blockIdx.x;
  if (smem_mode) {
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
    __syncthreads();
  }
  const uint64_t lo = (uint64_t)g * per, hi = min(n, lo + per);
  bool bad = false;
  for (uint64_t i0 = lo + threadIdx.x; i0 < hi; i0 += (uint64_t)kHistUnroll * blockDim.x) {
    int32_t r[kHistUnroll];
#pragma unroll
    for (int k = 0; k < kHistUnroll; ++k) {
      const uint64_t i = i0 + (uint64_t)k * blockDim.x;
      r[k] = i < hi ? rid(i) : 0;
    }
#pragma unroll
    for (int k = 0; k < kHistUnroll; ++k) {
      const uint64_t i = i0 + (uint64_t)k * blockDim.x;
      if (i < hi) {
        if (compact) compact[i] = r[k];
        if ((uint32_t)r[k] >= n_src) {
          bad = true;
        } else {
          const uint32_t b = (uint32_t)r[k] >> seg_log2;
          if (smem_mode) atomicAdd(&h[b], 1u);
          else atomicAdd(&tot[b], 1u);
        }
      }
    }
  }
  if (bad) atomicOr(err, ERR_RANGE);
  if (smem_mode) {
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) cnt[(uint64_t)g * nb + b] = h[b];
  }
}

// --------------------------------------------------------------------- K4
// CTA g re-reads the rids of [g*per, (g+1)*per) and appends each one's offset
// inside its segment to that segment's run at the CTA's cursor.  SLOT: the
// 3-pass plan records slot[i] = run position of rid i; otherwise the 2-pass
// plan records dest[pos] = i.  The entries one CTA adds to a run occupy the
// contiguous range the scan reserved for it; their order inside that range is
// not fixed (the result does not depend on it: every entry carries its slot).
template <class Rid, typename LoT, bool SLOT>
__global__ void __launch_bounds__(kPhaseThreads)
    k_distribute(Rid rid, uint64_t n, uint32_t seg_log2, uint32_t nb, uint32_t G, uint64_t per,
                 uint32_t* __restrict__ cur_g, LoT* __restrict__ lo_out, uint32_t* __restrict__ side,
                 const int* err, int smem_mode) {
  extern __shared__ uint32_t cur[];
  if (__syncthreads_or(threadIdx.x == 0 && error_set(err))) return;
  const uint32_t g = blockIdx.x;
  if (smem_mode) {
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) cur[b] = cur_g[(uint64_t)g * nb + b];
    __syncthreads();
  }
  const uint64_t lo = (uint64_t)g * per, hi = min(n, lo + per);
  const uint32_t mask = (1u << seg_log2) - 1u;
  for (uint64_t i0 = lo + threadIdx.x; i0 < hi; i0 += (uint64_t)kHistUnroll * blockDim.x) {
    int32_t r[kHistUnroll];
#pragma unroll
    for (int k = 0; k < kHistUnroll; ++k) {
      const uint64_t i = i0 + (uint64_t)k * blockDim.x;
      r[k] = i < hi ? rid(i) : 0;
    }
#pragma unroll
    for (int k = 0; k < kHistUnroll; ++k) {
      const uint64_t i = i0 + (uint64_t)k * blockDim.x;
      if (i < hi) {
        const uint32_t rv = (uint32_t)r[k];
        const uint32_t b = rv >> seg_log2;
        const uint32_t pos = smem_mode ? atomicAdd(&cur[b], 1u) : atomicAdd(&cur_g[b], 1u);
        lo_out[pos] = (LoT)(rv & mask);
        if (SLOT) side[i] = pos;
        else side[pos] = (uint32_t)i;
      }
    }
  }
}

// ------------------------------------------------------------------ K5/K7
// Persistent CTAs take work items (segment b, chunk c) from a global counter.
// A new segment is copied into shared memory with cp.async.bulk (16-byte
// aligned source) or with plain vector loads.  The chunk's run entries are
// then served kProbeSub at a time: their in-segment offsets (and, 2-pass,
// destination slots) are staged in shared memory while the bulk copy is in
// flight, and word w of entry k is copied from the segment to out[k]
// (INTERNAL staging, 3-pass, written as one contiguous stream in 16-byte
// vectors) or to out[dest[k]] (the destination, 2-pass).
constexpr uint32_t kProbeSub = 1024;

__device__ __forceinline__ uint4 pack16(const uint32_t (&x)[4]) { return make_uint4(x[0], x[1], x[2], x[3]); }
__device__ __forceinline__ uint4 pack16(const uint2 (&x)[2]) { return make_uint4(x[0].x, x[0].y, x[1].x, x[1].y); }

template <int WB, typename LoT>
__device__ __forceinline__ typename WordT<WB>::T probe_word(const typename WordT<WB>::T* sw, const LoT* lo_s,
                                                             uint32_t q, uint32_t w, uint32_t W) {
  return sw[(uint32_t)lo_s[q] * W + w];
}

template <int WB, typename LoT, bool SCATTER, bool PK = false>
__global__ void __launch_bounds__(kProbeThreads)
    k_probe(const uint8_t* __restrict__ src, uint32_t n_src, uint32_t rec, uint32_t seg_log2,
            const uint32_t* __restrict__ off, const uint32_t* __restrict__ itemoff, uint32_t nb, uint32_t chunk,
            const LoT* __restrict__ lo, const uint32_t* __restrict__ dest, uint8_t* __restrict__ out, uint32_t W,
            FastDiv fdW, int* err, uint32_t* item_counter, int use_bulk, uint32_t seg_smem, uint32_t pk_off = 0) {
  using T = typename WordT<WB>::T;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_item, s_b;
  uint8_t* seg = smem;
  LoT* lo_s = reinterpret_cast<LoT*>(smem + seg_smem);
  uint32_t* dest_s = reinterpret_cast<uint32_t*>(smem + seg_smem + kProbeSub * sizeof(LoT));
  if (__syncthreads_or(threadIdx.x == 0 && error_set(err))) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t n_items = itemoff[nb];
  uint32_t phase = 0;
  int64_t loaded = -1;
  const T* sw = reinterpret_cast<const T*>(seg);
  T* ow = reinterpret_cast<T*>(out);
  for (;;) {
    if (threadIdx.x == 0) {
      // once any CTA has raised an error no further item is taken, so no
      // further bulk copy is issued
      const uint32_t it = error_set(err) ? n_items : atomicAdd(item_counter, 1u);
      s_item = it;
      if (it < n_items) {
        uint32_t a = 0, z = nb;  // first j with itemoff[j] > it; itemoff[0] = 0 <= it
        while (a < z) {
          const uint32_t m = (a + z) >> 1;
          if (itemoff[m] > it) z = m;
          else a = m + 1;
        }
        s_b = a - 1;
      }
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= n_items) break;
    const uint32_t b = s_b;
    bool wait_bulk = false;
    if ((int64_t)b != loaded) {
      const uint64_t first = (uint64_t)b << seg_log2;
      const uint64_t left = (uint64_t)n_src - first;
      const uint32_t nrec = (uint32_t)(left < (1ull << seg_log2) ? left : (1ull << seg_log2));
      const uint32_t bytes = nrec * rec;
      const uint8_t* gsrc = src + first * rec;
      if (use_bulk) {
        const uint32_t body = bytes & ~15u;
        if (threadIdx.x == 0 && body) {
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&bar, body);
          for (uint32_t o = 0; o < body; o += kBulkPiece) bulk_g2s(seg + o, gsrc + o, min(kBulkPiece, body - o), &bar);
        }
        for (uint32_t o = body + threadIdx.x; o < bytes; o += blockDim.x) seg[o] = gsrc[o];
        wait_bulk = body != 0;
      } else {
        const T* gw = reinterpret_cast<const T*>(gsrc);
        T* sd = reinterpret_cast<T*>(seg);
        for (uint32_t o = threadIdx.x; o < bytes / WB; o += blockDim.x) sd[o] = gw[o];
      }
      loaded = b;
    }
    const uint32_t p0 = off[b] + (item - itemoff[b]) * chunk;
    const uint32_t p1 = min(off[b + 1], p0 + chunk);
    for (uint32_t q0 = p0; q0 < p1; q0 += kProbeSub) {
      const uint32_t nq = min(kProbeSub, p1 - q0);
      for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
        lo_s[q] = lo[q0 + q];
        if (SCATTER) dest_s[q] = dest[q0 + q];
      }
      if (wait_bulk) {
        // The copy is this CTA's own global -> shared bulk copy of at most
        // 104 KB, which lands within microseconds on a working device; the
        // bound only guards against a device that has stopped.  If it runs
        // out, thread 0 records the timeout and waits once more (bounded
        // again) for the copy already issued, so that the CTA does not
        // release shared memory the copy may still write; no other copy is
        // issued after the error bit is set (see the item claim above).
        const bool ok = mbar_wait_bounded(&bar, phase, kWaitCycles);
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0) {
            atomicOr(err, ERR_TIMEOUT);
            mbar_wait_bounded(&bar, phase, 4 * kWaitCycles);
          }
          return;
        }
        phase ^= 1u;
        wait_bulk = false;
      }
      __syncthreads();
      if constexpr (PK) {
        // join (§4.2.1, DPG-move): the dimension row of run entry q must carry
        // its own row number as its int64 little-endian key at pk_off
        bool bad = false;
        const bool pk8 = (rec % 8 == 0) && (pk_off % 8 == 0);
        for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
          const uint32_t l = lo_s[q];
          const uint8_t* pr = seg + (uint64_t)l * rec + pk_off;
          uint64_t v = 0;
          if (pk8) {
            v = *reinterpret_cast<const uint64_t*>(pr);
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v |= (uint64_t)pr[j] << (8 * j);
          }
          if (v != (((uint64_t)b << seg_log2) + l)) bad = true;
        }
        if (bad) atomicOr(err, ERR_RANGE);
      }
      const uint64_t total = (uint64_t)nq * W;
      if constexpr (SCATTER || WB >= 16 || WB <= 2) {
        for (uint64_t t = threadIdx.x; t < total; t += blockDim.x) {
          const uint32_t q = (uint32_t)fdiv(t, fdW);
          const uint32_t w = (uint32_t)(t - (uint64_t)q * W);
          const T v = probe_word<WB>(sw, lo_s, q, w, W);
          if (SCATTER) ow[(uint64_t)dest_s[q] * W + w] = v;
          else ow[(uint64_t)(q0 + q) * W + w] = v;
        }
      } else {
        // contiguous output: 16-byte vectors of VEC words, scalar head and tail
        constexpr uint32_t VEC = 16 / WB;
        const uint64_t g0 = (uint64_t)q0 * W, g1 = g0 + total;
        const uint64_t v0 = (g0 + VEC - 1) / VEC, v1 = g1 / VEC;
        const uint64_t head_end = v0 * VEC < g1 ? v0 * VEC : g1;
        for (uint64_t g = g0 + threadIdx.x; g < head_end; g += blockDim.x) {
          const uint32_t q = (uint32_t)fdiv(g - g0, fdW);
          ow[g] = probe_word<WB>(sw, lo_s, q, (uint32_t)(g - g0 - (uint64_t)q * W), W);
        }
        for (uint64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
          const uint64_t rel = v * VEC - g0;
          uint32_t q = (uint32_t)fdiv(rel, fdW);
          uint32_t w = (uint32_t)(rel - (uint64_t)q * W);
          T x[VEC];
#pragma unroll
          for (uint32_t j = 0; j < VEC; ++j) {
            x[j] = probe_word<WB>(sw, lo_s, q, w, W);
            if (++w == W) {
              w = 0;
              ++q;
            }
          }
          reinterpret_cast<uint4*>(out)[v] = pack16(x);
        }
        const uint64_t tail_start = v1 * VEC > head_end ? v1 * VEC : head_end;
        for (uint64_t g = tail_start + threadIdx.x; g < g1; g += blockDim.x) {
          const uint32_t q = (uint32_t)fdiv(g - g0, fdW);
          ow[g] = probe_word<WB>(sw, lo_s, q, (uint32_t)(g - g0 - (uint64_t)q * W), W);
        }
      }
      fence_proxy_async_smem();  // order this CTA's shared-memory accesses before the next bulk copy
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------- join rows
// out row r = A-part || B-part: wa words of row ia(r) of table A, then wb
// words of row ib(r) of table B, written as one coalesced word stream.
// CHECK_B: ib(r) must be below nrows_b (else the range bit, row skipped).
// pk_check: the int64 little-endian key at byte pk_off of the B row must equal
// ib(r) (else the range bit).
struct RowIdentity {
  __device__ __forceinline__ uint64_t operator()(uint64_t r) const { return r; }
};
struct RowSlot {
  const uint32_t* p;
  __device__ __forceinline__ uint64_t operator()(uint64_t r) const { return __ldg(p + r); }
};
struct RowField {  // int32 field of strided rows (a foreign-key column)
  const uint8_t* base;
  uint32_t stride;
  __device__ __forceinline__ uint64_t operator()(uint64_t r) const {
    return (uint64_t)(uint32_t)__ldg(reinterpret_cast<const int32_t*>(base + r * stride));
  }
};
struct RowPairKey {  // big-endian key bytes [0, kb) of sorted 8-byte pair r (kb <= 4)
  const uint8_t* pairs;
  uint32_t kb;
  __device__ __forceinline__ uint64_t operator()(uint64_t r) const {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(pairs + r * 8));
    return (uint64_t)(__byte_perm(w, 0, 0x0123) >> (8 * (4 - kb)));
  }
};

// U words per thread per step; MINB CTAs per SM asked of the compiler (0:
// none; its own choice is 53 registers and four CTAs at U = 8).  Measured
// on the 2e8-row join: DPG-move rows (key = an INTERNAL slot) 6.84 ms at
// U = 8 unbounded against 7.80 ms at U = 4 with eight CTAs per SM; direct
// rows (key = the fact row's fk, then a random dimension row) 6.31 ms at
// U = 4 with eight CTAs per SM against 8.94 ms at U = 8 unbounded.
template <int WB, class IA, class IB, bool CHECK_B, int U, int MINB>
__global__ void __launch_bounds__(kGatherThreads, MINB)
    k_join_rows(const uint8_t* __restrict__ ta, IA ia, uint32_t wa, const uint8_t* __restrict__ tb, IB ib,
                uint32_t wb, uint64_t nrows_b, uint8_t* __restrict__ out, uint64_t n, FastDiv fd_row,
                uint32_t pk_off, int pk_check, int* err) {
  using T = typename WordT<WB>::T;
  if (!CHECK_B && error_set(err)) return;
  const T* a = reinterpret_cast<const T*>(ta);
  const T* bt = reinterpret_cast<const T*>(tb);
  T* o = reinterpret_cast<T*>(out);
  const uint32_t row_w = wa + wb;
  const uint64_t total = n * row_w;
  const uint64_t step = (uint64_t)gridDim.x * kGatherThreads * U;
  const uint32_t pk_w0 = pk_off / WB, pk_w1 = (pk_off + 8 + WB - 1) / WB;
  // word t = row r, word w of the row, walked in steps of kGatherThreads words
  const uint32_t qs = (uint32_t)fdiv(kGatherThreads, fd_row), rs = kGatherThreads - qs * row_w;
  bool bad = false;
  for (uint64_t base = (uint64_t)blockIdx.x * kGatherThreads * U + threadIdx.x; base < total;
       base += step) {
    T v[U];
    bool ok[U];
    uint64_t r = fdiv(base, fd_row);
    uint32_t w = (uint32_t)(base - r * row_w);
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint64_t t = base + (uint64_t)k * kGatherThreads;
      ok[k] = false;
      if (t < total) {
        if (w < wa) {
          v[k] = a[ia(r) * wa + w];
          ok[k] = true;
        } else {
          const uint64_t key = ib(r);
          const uint32_t wbw = w - wa;
          if (!CHECK_B || key < nrows_b) {
            v[k] = bt[key * wb + wbw];
            ok[k] = true;
            if (pk_check && wbw >= pk_w0 && wbw < pk_w1 && !pk_word_ok<WB>(v[k], wbw, pk_off, key)) bad = true;
          } else {
            bad = true;
          }
        }
      }
      r += qs;
      w += rs;
      if (w >= row_w) {
        w -= row_w;
        ++r;
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (ok[k]) o[base + (uint64_t)k * kGatherThreads] = v[k];
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

template <class IA, class IB, bool CHECK_B, int U, int MINB>
void launch_join_rows(dpg_ctx& ctx, const char* name, uint32_t WB, const uint8_t* ta, IA ia, uint32_t a_bytes,
                      const uint8_t* tb, IB ib, uint32_t b_bytes, uint64_t nrows_b, uint8_t* out, uint64_t n,
                      uint32_t pk_off, int pk_check, cudaStream_t st) {
  const uint32_t wa = a_bytes / WB, wb = b_bytes / WB;
  const FastDiv f = make_fastdiv(wa + wb);
  const uint64_t total = n * (wa + wb);
  const uint64_t per_block = (uint64_t)kGatherThreads * U;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((total + per_block - 1) / per_block,
                                                                  (uint64_t)ctx.sms * 8));
  TraceScope ts(ctx, name, st);
#define DPG_JOIN(WBV)                                                                                           \
  k_join_rows<WBV, IA, IB, CHECK_B, U, MINB><<<grid, kGatherThreads, 0, st>>>(ta, ia, wa, tb, ib, wb, nrows_b, out, \
                                                                              n, f, pk_off, pk_check, ctx.d_err)
  switch (WB) {
    case 16: DPG_JOIN(16); break;
    case 8: DPG_JOIN(8); break;
    case 4: DPG_JOIN(4); break;
    case 2: DPG_JOIN(2); break;
    default: DPG_JOIN(1); break;
  }
#undef DPG_JOIN
  ctx.launches++;
}

// Sets the range bit when n > 0 rids address an empty source table.
__global__ void k_flag_range(int* err) { atomicOr(err, ERR_RANGE); }

// dpg_check_wait: one thread waits for *flag to become non-zero under the
// context's limit and records the timeout when it runs out.
__global__ void k_wait_check(const uint32_t* flag, int* err, long long limit) {
  bool ok;
  wait_word_bounded(flag, limit, &ok, [](uint32_t x) { return x != 0; });
  if (!ok) atomicOr(err, ERR_TIMEOUT);
}

// ------------------------------------------------------------------ host side

// CTAs per SM of the grid-stride gathers: records under 64 bytes run best
// with the SMs oversubscribed (32 CTAs per SM: 1.39 ms against 1.63 ms for one
// resident wave at 16 bytes), larger records with exactly one resident wave
// (0.47 against 0.56 ms at 100 bytes), measured on the 1e9-byte permutation
// workloads; DPG_GATHER_CTAS overrides.
template <class K>
uint64_t gather_grid(const dpg_ctx& ctx, K kern, uint32_t rec, uint64_t want) {
  const int knob = env_int("DPG_GATHER_CTAS", 0);
  const int per_sm = knob > 0 ? knob : (rec < 64 ? 32 : resident_per_sm(kern, kGatherThreads, 0));
  return std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx.sms * per_sm));
}

template <class Idx, bool CHECK>
void launch_gather(dpg_ctx& ctx, uint32_t WB, const uint8_t* src, uint8_t* dst, Idx idx, uint64_t n, uint32_t rec,
                   uint32_t n_src, cudaStream_t st, const char* name = nullptr) {
  const uint32_t W = rec / WB;
  const FastDiv f = make_fastdiv(W);
  const uint64_t total = n * W;
  TraceScope ts(ctx, name ? name : (CHECK ? "k_gather_direct" : "k_gather_phase3"), st);
  if ((WB == 4 || WB == 8) && W >= 16 / WB && reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
    const uint64_t per_block = (uint64_t)kGatherThreads * kGather16Unroll;
    const uint64_t want = (total / (16 / WB) + per_block - 1) / per_block;
    auto kern = WB == 4 ? k_gather16<4, CHECK, Idx> : k_gather16<8, CHECK, Idx>;
    const int grid = (int)gather_grid(ctx, kern, rec, want);
    kern<<<grid, kGatherThreads, 0, st>>>(src, dst, idx, n, W, f, n_src, ctx.d_err);
    ctx.launches++;
    return;
  }
  const uint64_t per_block = (uint64_t)kGatherThreads * kGatherUnroll;
  const uint64_t want = (total + per_block - 1) / per_block;
  auto kern = WB == 16  ? k_gather<16, CHECK, Idx>
              : WB == 8 ? k_gather<8, CHECK, Idx>
              : WB == 4 ? k_gather<4, CHECK, Idx>
              : WB == 2 ? k_gather<2, CHECK, Idx>
                        : k_gather<1, CHECK, Idx>;
  const int grid = (int)gather_grid(ctx, kern, rec, want);
  kern<<<grid, kGatherThreads, 0, st>>>(src, dst, idx, n, W, f, n_src, ctx.d_err);
  ctx.launches++;
}

}  // namespace

void launch_slot_gather(dpg_ctx& ctx, uint32_t wb, const uint8_t* src, uint8_t* dst, const uint32_t* slot,
                        uint64_t n, uint32_t rec, uint32_t n_src, cudaStream_t st, const char* name) {
  launch_gather<SlotArray, false>(ctx, wb, src, dst, SlotArray{slot}, n, rec, n_src, st, name);
}

void launch_join_phase3(dpg_ctx& ctx, const Retrieval& r, const uint8_t* stage, const uint32_t* slot) {
  const JoinSpec& j = *r.join;
  const uint32_t wb = std::min({pow2_align(j.fact_bytes), pow2_align(j.dim_bytes),
                                pow2_align(reinterpret_cast<uintptr_t>(j.out)),
                                pow2_align(reinterpret_cast<uintptr_t>(j.fact)),
                                pow2_align(reinterpret_cast<uintptr_t>(j.dim))});
  if (j.mode == 0)
    launch_join_rows<RowIdentity, RowSlot, false, 8, 0>(ctx, "k_join_move_rows", wb, j.fact, RowIdentity{},
                                                        j.fact_bytes, stage, RowSlot{slot}, j.dim_bytes, j.n_dim,
                                                        j.out, r.n, j.pk_off, 0, r.stream);
  else
    launch_join_rows<RowSlot, RowPairKey, false, 8, 0>(ctx, "k_join_sort_rows", wb, stage, RowSlot{slot},
                                                       j.fact_bytes, j.dim, RowPairKey{j.sorted_pairs, j.key_bytes},
                                                       j.dim_bytes, j.n_dim, j.out, r.n, j.pk_off, 1, r.stream);
}

namespace {

template <typename LoT, bool SCATTER, bool PK = false>
void launch_probe(dpg_ctx& ctx, uint32_t WB, const Retrieval& r, uint32_t seg_log2, const uint32_t* off,
                  const uint32_t* itemoff, uint32_t nb, uint32_t chunk, const LoT* lo, const uint32_t* dest,
                  uint8_t* out, uint32_t* counter, int use_bulk, size_t seg_smem, uint32_t pk_off = 0) {
  const uint32_t W = r.rec / WB;
  const size_t smem = seg_smem + kProbeSub * sizeof(LoT) + (SCATTER ? kProbeSub * 4 : 0);
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (smem + 1024 + 256)));
  const FastDiv f = make_fastdiv(W);
  const int grid = ctx.sms * per_sm;
  TraceScope ts(ctx, SCATTER ? "k_probe_scatter" : "k_probe", r.stream);
#define DPG_PROBE(WBV)                                                                                         \
  {                                                                                                            \
    auto kern = k_probe<WBV, LoT, SCATTER, PK>;                                                                \
    set_smem(kern, smem);                                                                                      \
    kern<<<grid, kProbeThreads, smem, r.stream>>>(r.src, (uint32_t)r.n_src, r.rec, seg_log2, off, itemoff, nb, \
                                                 chunk, lo, dest, out, W, f, ctx.d_err, counter, use_bulk,     \
                                                 (uint32_t)seg_smem, pk_off);                                  \
  }
  switch (WB) {
    case 16: DPG_PROBE(16) break;
    case 8: DPG_PROBE(8) break;
    case 4: DPG_PROBE(4) break;
    case 2: DPG_PROBE(2) break;
    default: DPG_PROBE(1) break;
  }
#undef DPG_PROBE
  ctx.launches++;
}


// Scratch layout of the shared-memory-segment plans (variants 2 and 3), each
// piece 256-byte aligned.
struct Layout3 {
  uint32_t sl, nb, grid, G, chunk;
  uint64_t S, per;
  bool smem_mode, three, strided;
  size_t b_cnt, b_psum, b_tot, b_off, b_ctr, b_lo, b_side, b_ts, b_rc, b_stage, need;
};

Layout3 layout3(const dpg_ctx& ctx, const Retrieval& r, const Plan& plan, size_t lo_size, bool strided) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  Layout3 L;
  L.sl = (uint32_t)plan.seg_log2;
  L.S = 1ull << L.sl;
  L.nb = (uint32_t)((r.n_src + L.S - 1) >> L.sl);
  L.smem_mode = L.nb <= kSmemBuckets;
  L.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)ctx.sms * 2, (r.n + 8191) / 8192));
  L.G = L.smem_mode ? L.grid : 1;
  L.per = (r.n + L.grid - 1) / L.grid;
  L.chunk = plan.chunk ? plan.chunk : (uint32_t)std::min<uint64_t>(4 * L.S, 1u << 20);
  L.three = plan.variant != 2 || r.join != nullptr;
  L.strided = strided;
  L.b_cnt = al((size_t)L.nb * L.G * 4);
  L.b_psum = al((size_t)L.nb * kScanSlices * 4);
  L.b_tot = al((size_t)L.nb * 4);
  L.b_off = al(((size_t)L.nb + 1) * 4);
  L.b_ctr = 256;
  L.b_lo = al(r.n * lo_size);
  L.b_side = al(r.n * 4);
  L.b_ts = al((size_t)((L.nb + kScanTile - 1) / kScanTile) * 4);
  L.b_rc = strided ? al(r.n * 4) : 0;  // rids copied out of strided pairs by Phase I pass 1
  L.b_stage = L.three ? al(r.n * r.rec) : 0;
  L.need = L.b_cnt + L.b_psum + L.b_tot + 2 * L.b_off + L.b_ctr + 2 * L.b_ts + L.b_lo + L.b_side + L.b_rc +
           L.b_stage;
  return L;
}

template <class Rid, typename LoT>
int run_dpg_t(dpg_ctx& ctx, const Retrieval& r, Rid rid, const Plan& plan) {
  const Layout3 L = layout3(ctx, r, plan, sizeof(LoT), !std::is_same<Rid, RidArray>::value);
  const uint32_t sl = L.sl, nb = L.nb, grid = L.grid, G = L.G, chunk = L.chunk;
  const uint64_t S = L.S, per = L.per;
  const bool smem_mode = L.smem_mode, three = L.three, strided = L.strided;
  const size_t b_cnt = L.b_cnt, b_psum = L.b_psum, b_tot = L.b_tot, b_off = L.b_off, b_ctr = L.b_ctr, b_lo = L.b_lo,
               b_side = L.b_side, b_ts = L.b_ts, b_rc = L.b_rc;
  if (int s = ensure_scratch(ctx, L.need)) return s;
  uint8_t* p = static_cast<uint8_t*>(ctx.scratch);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(p); p += b_cnt;
  uint32_t* psum = reinterpret_cast<uint32_t*>(p); p += b_psum;
  uint32_t* tot = reinterpret_cast<uint32_t*>(p); p += b_tot;
  uint32_t* off = reinterpret_cast<uint32_t*>(p); p += b_off;
  uint32_t* itemoff = reinterpret_cast<uint32_t*>(p); p += b_off;
  uint32_t* counter = reinterpret_cast<uint32_t*>(p); p += b_ctr;
  uint32_t* tsum = reinterpret_cast<uint32_t*>(p); p += b_ts;
  uint32_t* isum = reinterpret_cast<uint32_t*>(p); p += b_ts;
  LoT* lo = reinterpret_cast<LoT*>(p); p += b_lo;
  uint32_t* side = reinterpret_cast<uint32_t*>(p); p += b_side;
  int32_t* rc = strided ? reinterpret_cast<int32_t*>(p) : nullptr; p += b_rc;
  uint8_t* stage = three ? p : nullptr;

  cudaError_t e = smem_mode ? cudaSuccess : cudaMemsetAsync(tot, 0, (size_t)nb * 4, r.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(tsum, 0, 2 * b_ts, r.stream);  // tsum, isum
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  const size_t phase_smem = smem_mode ? (size_t)nb * 4 : 0;
  {
    TraceScope ts(ctx, "k_hist", r.stream);
    auto kern = k_hist<Rid>;
    set_smem(kern, phase_smem);
    kern<<<grid, kPhaseThreads, phase_smem, r.stream>>>(rid, r.n, (uint32_t)r.n_src, sl, nb, G, per, cnt, tot,
                                                        ctx.d_err, smem_mode, rc);
    ctx.launches++;
  }
  {
    TraceScope ts(ctx, "k_bucket_totals", r.stream);
    k_bucket_totals<<<(nb + kScanBlock - 1) / kScanBlock, 1024, 0, r.stream>>>(cnt, tot, psum, nb, G, chunk,
                                                                               tsum, isum, ctx.d_err, smem_mode);
  }
  {
    TraceScope ts(ctx, "k_scan", r.stream);
    k_scan<<<(nb + kScanBlock - 1) / kScanBlock, 1024, 0, r.stream>>>(tot, psum, tsum, isum, nb, G, chunk, cnt,
                                                                      off, itemoff, counter, ctx.d_err, smem_mode);
  }
  ctx.launches += 2;
  {
    TraceScope ts(ctx, "k_distribute", r.stream);
    const RidArray ra{strided ? rc : reinterpret_cast<const int32_t*>(r.rids.base)};
    auto kern = three ? k_distribute<RidArray, LoT, true> : k_distribute<RidArray, LoT, false>;
    set_smem(kern, phase_smem);
    kern<<<grid, kPhaseThreads, phase_smem, r.stream>>>(ra, r.n, sl, nb, G, per, cnt, lo, side, ctx.d_err,
                                                        smem_mode);
    ctx.launches++;
  }
  // Phase II: word size limited by the record size, the shared-memory record
  // offsets, and the output base (staging is 256-byte aligned).
  const uintptr_t src_a = reinterpret_cast<uintptr_t>(r.src);
  const uint32_t seg_bytes = (uint32_t)(std::min<uint64_t>(S, r.n_src) * r.rec);
  const int use_bulk = (src_a % 16 == 0) && ((S * r.rec) % 16 == 0);
  uint32_t wb_probe = pow2_align(r.rec);
  if (!three) wb_probe = std::min(wb_probe, pow2_align(reinterpret_cast<uintptr_t>(r.dst)));
  if (!use_bulk) wb_probe = std::min(wb_probe, pow2_align(src_a));
  const size_t probe_smem = ((size_t)seg_bytes + 15) & ~size_t(15);
  if (r.join && r.join->mode == 0)
    launch_probe<LoT, false, true>(ctx, wb_probe, r, sl, off, itemoff, nb, chunk, lo, nullptr, stage, counter,
                                   use_bulk, probe_smem, r.join->pk_off);
  else if (three)
    launch_probe<LoT, false>(ctx, wb_probe, r, sl, off, itemoff, nb, chunk, lo, nullptr, stage, counter, use_bulk,
                             probe_smem);
  else
    launch_probe<LoT, true>(ctx, wb_probe, r, sl, off, itemoff, nb, chunk, lo, side, r.dst, counter, use_bulk,
                            probe_smem);
  if (r.join) {
    launch_join_phase3(ctx, r, stage, side);
  } else if (three) {
    // Phase III
    const uint32_t wb = std::min(pow2_align(r.rec), pow2_align(reinterpret_cast<uintptr_t>(r.dst)));
    launch_gather<SlotArray, false>(ctx, wb, stage, r.dst, SlotArray{side}, r.n, r.rec, (uint32_t)r.n_src,
                                    r.stream);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "dpg launch");
  return DPG_OK;
}



}  // namespace

namespace {

int smem_seg_log2(const Retrieval& r) {
  int sl = 0;
  while (sl < 30 && ((2ull << sl) * r.rec) <= kSegBytesMax) ++sl;
  return sl;
}

// Runs of about run_bytes of source for the L2-run plan, at most kL2MaxRuns.
int l2_seg_log2(const Retrieval& r, uint64_t run_bytes) {
  int k = 0;
  while (k < 31 && ((2ull << k) * r.rec) <= run_bytes) ++k;
  while (k < 31 && ((r.n_src + (1ull << k) - 1) >> k) > kL2MaxRuns) ++k;
  return k;
}

int ilog2(uint64_t x) {
  int k = 0;
  while (x >>= 1) ++k;
  return k;
}

}  // namespace

uint64_t plan_key(const Retrieval& r) {
  return ((uint64_t)r.rec << 32) | ((uint64_t)ilog2(r.n_src + 1) << 24) | ((uint64_t)ilog2(r.n + 1) << 16) |
         ((uint64_t)(r.rids.stride != 4) << 8) | (uint64_t)(r.join != nullptr);
}

Plan choose_plan(const dpg_ctx& ctx, const Retrieval& r) {
  Plan p;
  p.seg_log2 = smem_seg_log2(r);
  p.variant = 3;
  const bool env = std::getenv("DPG_VARIANT") || std::getenv("DPG_SEG_LOG2") || std::getenv("DPG_L2_RUN_KB");
  if (!env && !r.join) {
    auto it = ctx.plans.find(plan_key(r));
    if (it != ctx.plans.end()) {
      p.variant = it->second.first;
      p.seg_log2 = it->second.second;
      return p;
    }
  }
  // Untuned default by record size, from the 1e9-byte permutation sweep
  // (16..128 B: L2 runs; 256 B: 2-pass shared-memory segments).  Joins, on
  // the 2e8-row Zipf workload (64-byte dimension rows): the DPG-sort join
  // moves fact rows like a retrieval (L2 runs: 24.0 against 27.6 ms); DPG-move
  // probes each dimension row about 20 times, and the L2-run plan's cheaper
  // Phase I (1.1 against 5.5 ms) outweighs its Phase II, whose hot rows come
  // from the L2 rather than shared memory (4.2 against 2.4 ms): 11.6 against
  // 14.9 ms.  Dimension rows of 192 bytes and more keep the 3-pass plan.
  // Forcing a segment size or chunk keeps the shared-memory plan.
  int dflt = r.rec < 192 ? 4 : 2;
  if (r.join) dflt = r.rec < 192 ? 4 : 3;
  if (std::getenv("DPG_SEG_LOG2") || std::getenv("DPG_CHUNK")) dflt = 3;
  p.variant = env_int("DPG_VARIANT", dflt);
  const int o = env_int("DPG_SEG_LOG2", -1);
  if (o >= 0 && (1ull << o) * r.rec <= kSegBytesMax) p.seg_log2 = o;
  p.chunk = (uint32_t)env_int("DPG_CHUNK", 0);
  if (r.join && p.variant == 2) p.variant = 3;  // joins need INTERNAL and a slot per row
  if (p.variant == 4) p.seg_log2 = l2_seg_log2(r, (uint64_t)env_int("DPG_L2_RUN_KB", 16384) << 10);
  return p;
}

std::vector<Plan> plan_candidates(const dpg_ctx& ctx, const Retrieval& r) {
  (void)ctx;
  std::vector<Plan> c;
  const int sl = smem_seg_log2(r);
  for (int d = 0; d <= 2; ++d)
    if (sl - d >= 0) {
      Plan p;
      p.variant = 3;
      p.seg_log2 = sl - d;
      c.push_back(p);
    }
  {
    Plan p;
    p.variant = 2;
    p.seg_log2 = sl;
    c.push_back(p);
  }
  for (uint64_t mb : {4ull, 8ull, 16ull}) {
    Plan p;
    p.variant = 4;
    p.seg_log2 = l2_seg_log2(r, mb << 20);
    if (((r.n_src + (1ull << p.seg_log2) - 1) >> p.seg_log2) <= kL2MaxRuns) c.push_back(p);
  }
  return c;
}

size_t retrieve_scratch_need(const dpg_ctx& ctx, const Retrieval& r) {
  if (r.n == 0 || r.n_src == 0) return 0;
  const Plan plan = choose_plan(ctx, r);
  const bool strided = r.rids.stride != 4;
  if (plan.variant == 4) return l2_scratch_need(ctx, r, plan, strided);
  return layout3(ctx, r, plan, plan.seg_log2 <= 16 ? 2 : 4, strided).need;
}

int run_dpg(dpg_ctx& ctx, const Retrieval& r, const Plan& plan) {
  if (r.n == 0) return DPG_OK;
  ctx.last_variant = plan.variant;
  ctx.last_seg_log2 = plan.seg_log2;
  if (r.n_src == 0) {
    k_flag_range<<<1, 1, 0, r.stream>>>(ctx.d_err);
    ctx.launches++;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DPG_OK : cuda_fail(ctx, e, "flag");
  }
  if (plan.variant == 4) return run_dpg_l2(ctx, r, plan);
  if ((1ull << plan.seg_log2) * r.rec > kSegBytesMax && plan.seg_log2 > 0) return DPG_EINVAL;
  const bool lo16 = plan.seg_log2 <= 16;
  if (r.rids.stride == 4) {
    RidArray a{reinterpret_cast<const int32_t*>(r.rids.base)};
    return lo16 ? run_dpg_t<RidArray, uint16_t>(ctx, r, a, plan) : run_dpg_t<RidArray, uint32_t>(ctx, r, a, plan);
  }
  RidStrided s{r.rids.base, r.rids.stride};
  return lo16 ? run_dpg_t<RidStrided, uint16_t>(ctx, r, s, plan) : run_dpg_t<RidStrided, uint32_t>(ctx, r, s, plan);
}

int launch_wait_check(dpg_ctx& ctx, const uint32_t* flag, cudaStream_t st) {
  TraceScope ts(ctx, "k_wait_check", st);
  k_wait_check<<<1, 1, 0, st>>>(flag, ctx.d_err, ctx.wait_cycles);
  ctx.launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DPG_OK : cuda_fail(ctx, e, "wait check launch");
}

int run_join_direct(dpg_ctx& ctx, const JoinSpec& j, uint64_t n_fact, cudaStream_t st) {
  if (n_fact == 0) return DPG_OK;
  const uint32_t wb = std::min({pow2_align(j.fact_bytes), pow2_align(j.dim_bytes),
                                pow2_align(reinterpret_cast<uintptr_t>(j.out)),
                                pow2_align(reinterpret_cast<uintptr_t>(j.fact)),
                                pow2_align(reinterpret_cast<uintptr_t>(j.dim))});
  launch_join_rows<RowIdentity, RowField, true, 4, 8>(ctx, "k_join_direct_rows", wb, j.fact, RowIdentity{},
                                                      j.fact_bytes, j.dim, RowField{j.fact + j.fk_off, j.fact_bytes},
                                                      j.dim_bytes, j.n_dim, j.out, n_fact, j.pk_off, 1, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DPG_OK : cuda_fail(ctx, e, "join direct launch");
}

int run_direct(dpg_ctx& ctx, const Retrieval& r) {
  if (r.n == 0) return DPG_OK;
  const uint32_t wb = std::min({pow2_align(r.rec), pow2_align(reinterpret_cast<uintptr_t>(r.src)),
                                pow2_align(reinterpret_cast<uintptr_t>(r.dst))});
  if (r.rids.stride == 4)
    launch_gather<RidArray, true>(ctx, wb, r.src, r.dst, RidArray{reinterpret_cast<const int32_t*>(r.rids.base)},
                                  r.n, r.rec, (uint32_t)r.n_src, r.stream);
  else
    launch_gather<RidStrided, true>(ctx, wb, r.src, r.dst, RidStrided{r.rids.base, r.rids.stride}, r.n, r.rec,
                                    (uint32_t)r.n_src, r.stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DPG_OK : cuda_fail(ctx, e, "direct launch");
}

}  // namespace dpg

// ---------------------------------------------------------------------------
// Allocation-free retrieval (dpg_retrieve_noalloc in include/dpg.h).
//
// Some callers cannot call cudaMalloc: code that runs while a caching
// allocator owns all free device memory, code inside a memory-capped or
// pre-budgeted region, or a plug-in loaded into a host process that forbids
// device allocations after start-up.  For them this entry point runs the
// 2-pass DPG plan (no INTERNAL staging table) with its scratch in one
// fixed-size __device__ array that the CUDA module reserves on every device
// the library is loaded on, for the life of the process.  It needs no
// context, allocates nothing, and calls no allocating routine.
//
// Capacity: at most kNoallocMaxRids rids, at most kNoallocMaxSegs source
// segments (about 420 MB of 100-byte records); larger requests return
// DPG_EINVAL before anything is enqueued.  Every call shares the array, so
// calls whose GPU work overlaps (two streams, two host threads) race.
namespace dpg {
namespace {

constexpr uint64_t kNoallocMaxRids = 1ull << 21;
constexpr uint32_t kNoallocMaxSegs = 4096;
constexpr uint32_t kNoallocMaxCtas = 304;
constexpr size_t kNaAl(size_t x) { return (x + 255) & ~size_t(255); }
// byte offsets inside the array
constexpr size_t kNaErr = 0;
constexpr size_t kNaCounter = 256;
constexpr size_t kNaTot = 512;
constexpr size_t kNaOff = kNaTot + kNaAl(kNoallocMaxSegs * 4);
constexpr size_t kNaItemoff = kNaOff + kNaAl((kNoallocMaxSegs + 1) * 4);
constexpr size_t kNaTsum = kNaItemoff + kNaAl((kNoallocMaxSegs + 1) * 4);
constexpr size_t kNaIsum = kNaTsum + 256;
constexpr size_t kNaCnt = kNaIsum + 256;
constexpr size_t kNaLo = kNaCnt + kNaAl((size_t)kNoallocMaxSegs * kNoallocMaxCtas * 4);
constexpr size_t kNaDest = kNaLo + kNaAl(kNoallocMaxRids * 2);
constexpr size_t kNaPsum = kNaDest + kNaAl(kNoallocMaxRids * 4);
constexpr size_t kNoallocBytes = kNaPsum + kNaAl((size_t)kNoallocMaxSegs * kScanSlices * 4);
static_assert((kNoallocMaxSegs + kScanTile - 1) / kScanTile * 4 <= 256, "tile sums fit their slot");

// The scratch itself: ~17.6 MB per device.  Host code must not use this name
// as an address (it is a host-side stand-in); it asks the runtime for the
// device address once per device instead.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kNoallocDevices] = {};
int g_noalloc_sms[kNoallocDevices] = {};

// Device address of the array for the current device, looked up on the first
// call made with that device current.  That lookup is also what makes the
// runtime load this file's device code on the device when nothing else of the
// library has run there yet (lazy module loading), and loading the module is
// when the array is reserved: the first call is the set-up call.
int noalloc_setup(int dev, unsigned char** out, int* sms) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return DPG_ECUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return DPG_ECUDA;
    }
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    g_noalloc_sms[dev] = n;
  }
  *out = g_noalloc_ptr[dev];
  *sms = g_noalloc_sms[dev];
  return DPG_OK;
}

template <class Launch>
int noalloc_probe(uint32_t wb, Launch&& go) {
  switch (wb) {
    case 16: go(std::integral_constant<int, 16>{}); break;
    case 8: go(std::integral_constant<int, 8>{}); break;
    case 4: go(std::integral_constant<int, 4>{}); break;
    case 2: go(std::integral_constant<int, 2>{}); break;
    default: go(std::integral_constant<int, 1>{}); break;
  }
  return DPG_OK;
}

}  // namespace
}  // namespace dpg

extern "C" dpg_status dpg_retrieve_noalloc(const void* src_v, size_t n_src, size_t rec, size_t n,
                                           const int32_t* rids, void* dst_v, void* stream_v) {
  using namespace dpg;
  if (rec == 0 || rec > kMaxDpgRecBytes || n_src > 0x7fffffffULL) return DPG_EINVAL;
  if (n == 0) return DPG_OK;
  if (!rids || !dst_v || (n_src > 0 && !src_v)) return DPG_EINVAL;
  if (n > kNoallocMaxRids) return DPG_EINVAL;
  const uint8_t* src = static_cast<const uint8_t*>(src_v);
  uint8_t* dst = static_cast<uint8_t*>(dst_v);
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(src), d0 = reinterpret_cast<uintptr_t>(dst),
                  r0 = reinterpret_cast<uintptr_t>(rids);
  if (n_src && s0 < d0 + n * rec && d0 < s0 + n_src * rec) return DPG_EINVAL;
  if (r0 < d0 + n * rec && d0 < r0 + n * 4) return DPG_EINVAL;
  int sl = 0;
  while (sl < 16 && ((2ull << sl) * rec) <= kSegBytesMax) ++sl;
  const uint64_t S = 1ull << sl;
  const uint32_t nb = (uint32_t)((n_src + S - 1) >> sl);
  if (nb > kNoallocMaxSegs) return DPG_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocDevices) {
    cudaGetLastError();
    return DPG_ECUDA;
  }
  unsigned char* base = nullptr;
  int sms = 0;
  if (int s = noalloc_setup(dev, &base, &sms)) return (dpg_status)s;
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  int* err = reinterpret_cast<int*>(base + kNaErr);
  uint32_t* counter = reinterpret_cast<uint32_t*>(base + kNaCounter);
  uint32_t* tot = reinterpret_cast<uint32_t*>(base + kNaTot);
  uint32_t* off = reinterpret_cast<uint32_t*>(base + kNaOff);
  uint32_t* itemoff = reinterpret_cast<uint32_t*>(base + kNaItemoff);
  uint32_t* tsum = reinterpret_cast<uint32_t*>(base + kNaTsum);
  uint32_t* isum = reinterpret_cast<uint32_t*>(base + kNaIsum);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + kNaCnt);
  uint16_t* lo = reinterpret_cast<uint16_t*>(base + kNaLo);
  uint32_t* dest = reinterpret_cast<uint32_t*>(base + kNaDest);
  uint32_t* psum = reinterpret_cast<uint32_t*>(base + kNaPsum);

  // the error word and the tile sums must start at zero on every call
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(tsum, 0, 512, st);  // tsum and isum, adjacent
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DPG_ECUDA;
  }
  if (n_src == 0) {
    k_flag_range<<<1, 1, 0, st>>>(err);
  } else {
    const uint32_t grid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>({(uint64_t)sms * 2, (uint64_t)kNoallocMaxCtas, (n + 8191) / 8192}));
    const uint64_t per = (n + grid - 1) / grid;
    const uint32_t chunk = (uint32_t)(4 * S);
    const size_t phase_smem = (size_t)nb * 4;
    RidArray rid{rids};
    auto kh = k_hist<RidArray>;
    set_smem(kh, phase_smem);
    kh<<<grid, kPhaseThreads, phase_smem, st>>>(rid, n, (uint32_t)n_src, sl, nb, grid, per, cnt, tot, err, 1,
                                                 nullptr);
    k_bucket_totals<<<(nb + kScanBlock - 1) / kScanBlock, 1024, 0, st>>>(cnt, tot, psum, nb, grid, chunk, tsum,
                                                                         isum, err, 1);
    k_scan<<<(nb + kScanBlock - 1) / kScanBlock, 1024, 0, st>>>(tot, psum, tsum, isum, nb, grid, chunk, cnt, off,
                                                                itemoff, counter, err, 1);
    auto kd = k_distribute<RidArray, uint16_t, false>;
    set_smem(kd, phase_smem);
    kd<<<grid, kPhaseThreads, phase_smem, st>>>(rid, n, sl, nb, grid, per, cnt, lo, dest, err, 1);
    const int use_bulk = (s0 % 16 == 0) && ((S * rec) % 16 == 0);
    uint32_t wb = std::min(pow2_align(rec), pow2_align(d0));
    if (!use_bulk) wb = std::min(wb, pow2_align(s0));
    const uint32_t seg_bytes = (uint32_t)(std::min<uint64_t>(S, n_src) * rec);
    const size_t probe_smem = ((size_t)seg_bytes + 15) & ~size_t(15);
    noalloc_probe(wb, [&](auto wbc) {
      constexpr int WBV = decltype(wbc)::value;
      auto kp = k_probe<WBV, uint16_t, true>;
      const size_t smem = probe_smem + kProbeSub * (2 + 4);
      set_smem(kp, smem);
      const uint32_t W = (uint32_t)rec / WBV;
      kp<<<sms * 2, kProbeThreads, smem, st>>>(src, (uint32_t)n_src, (uint32_t)rec, sl, off, itemoff, nb, chunk,
                                                lo, dest, dst, W, make_fastdiv(W), err, counter, use_bulk,
                                                (uint32_t)probe_smem, 0u);
    });
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&bits, g_noalloc_scratch, sizeof(int), kNaErr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DPG_ECUDA;
  }
  if (bits & ERR_RANGE) return DPG_ERANGE;
  if (bits & ERR_TIMEOUT) return DPG_ETIMEOUT;
  return DPG_OK;
}
