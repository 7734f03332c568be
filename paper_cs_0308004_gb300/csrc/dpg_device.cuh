// Device-side helpers shared by the record-retrieval kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpg {

// Bits of the context's device error word.
enum : int { ERR_RANGE = 1, ERR_TIMEOUT = 2 };

// Bounded device-side waits give up after this many SM clock cycles unless
// the context sets another limit (about 1 s at the 2.07 GHz SM clock).
constexpr long long kWaitCycles = 2000000000LL;

// q = n / d by a 64-bit multiply-high with m = ceil(2^64 / d) = (2^64 + e) / d,
// 0 <= e < d.  Then n * m / 2^64 = n / d + n * e / (d * 2^64), and the floor
// is exact whenever n * e < 2^64, so whenever n * d < 2^64.  The launches
// divide word indices t < n * W by W = rec / WB (n < 2^31, W <= 2^16: t * W
// < 2^63) and join-row word indices by the row's word count, for which the
// join entry point checks the bound.  make_fastdiv(d, n_end) states the
// largest dividend + 1 a launch will use and reports, in `exact`, whether
// every n < n_end divides exactly; launches refuse to run when it does not.
// d == 1 is handled apart because m would be 2^64.
struct FastDiv {
  uint64_t m;
  uint32_t d;
};

inline bool fastdiv_exact(uint32_t d, uint64_t n_end) { return d <= 1 || n_end <= UINT64_MAX / d; }

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.m = (d <= 1) ? 0 : (UINT64_MAX / d + 1);
  return f;
}

__device__ __forceinline__ uint64_t fdiv(uint64_t n, const FastDiv& f) {
  return f.d == 1 ? n : __umul64hi(n, f.m);
}

// The unit in which a kernel moves record bytes: WB bytes, WB a power of two
// that divides the record size and every base address involved.
template <int WB> struct WordT;
template <> struct WordT<16> { using T = uint4; };
template <> struct WordT<8> { using T = uint2; };
template <> struct WordT<4> { using T = uint32_t; };
template <> struct WordT<2> { using T = uint16_t; };
template <> struct WordT<1> { using T = uint8_t; };

// The key check of the joins (§4.2.1): a dimension row must carry its own row
// number as the int64 little-endian key at byte pk_off.  Word w of the row
// (WB bytes at byte w*WB, overlapping that key: -8 < pk_off - w*WB < WB) is
// checked by comparing its bytes, as two 64-bit halves, with the key shifted
// to its place in the word, under the mask of the bytes the two share.
template <int WB>
__host__ __device__ __forceinline__ void word_halves(const typename WordT<WB>::T& v, uint64_t& lo, uint64_t& hi) {
  if constexpr (WB == 16) {
    lo = v.x | (uint64_t)v.y << 32;
    hi = v.z | (uint64_t)v.w << 32;
  } else if constexpr (WB == 8) {
    lo = v.x | (uint64_t)v.y << 32;
    hi = 0;
  } else {
    lo = v;
    hi = 0;
  }
}

template <int WB>
__host__ __device__ __forceinline__ bool pk_word_ok(const typename WordT<WB>::T& v, uint32_t w, uint32_t pk_off,
                                                    uint64_t key) {
  uint64_t lo, hi;
  word_halves<WB>(v, lo, hi);
  const int s = (int)pk_off - (int)(w * WB);  // key byte b is byte s + b of the word
  uint64_t klo, khi, mlo, mhi;
  if (s <= 0) {
    klo = key >> (-8 * s);
    mlo = ~0ull >> (-8 * s);
    khi = mhi = 0;
  } else if (s < 8) {
    klo = key << (8 * s);
    mlo = ~0ull << (8 * s);
    khi = key >> (64 - 8 * s);
    mhi = ~0ull >> (64 - 8 * s);
  } else {
    klo = mlo = 0;
    khi = key << (8 * (s - 8));
    mhi = ~0ull << (8 * (s - 8));
  }
  if constexpr (WB < 8) mlo &= (1ull << (8 * WB)) - 1;
  if constexpr (WB <= 8) mhi = 0;
  return ((lo ^ klo) & mlo) == 0 && ((hi ^ khi) & mhi) == 0;
}

// Rid sources: a plain int32 array, or the int32 field of strided
// key-pointer pairs.  Both address 4-byte-aligned int32 values.
struct RidArray {
  const int32_t* p;
  __device__ __forceinline__ int32_t operator()(uint64_t i) const { return __ldg(p + i); }
};
struct RidStrided {
  const uint8_t* base;  // points at the rid field of pair 0
  uint32_t stride;
  __device__ __forceinline__ int32_t operator()(uint64_t i) const {
    return __ldg(reinterpret_cast<const int32_t*>(base + i * stride));
  }
};
struct SlotArray {
  const uint32_t* p;
  __device__ __forceinline__ int32_t operator()(uint64_t i) const { return (int32_t)__ldg(p + i); }
};

__device__ __forceinline__ bool error_set(const int* err) {
  return *reinterpret_cast<const volatile int*>(err) != 0;
}

// ---- mbarrier + bulk copy (inline PTX, sm_90 and later) --------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy completing on `bar`; dst, src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Asynchronous global -> shared copies of B = 4, 8 or 16 bytes (both
// addresses B-aligned); cp_async_wait_all() waits for all of this thread's.
template <int B> __device__ __forceinline__ void cp_async(void* smem, const void* gmem);
template <> __device__ __forceinline__ void cp_async<16>(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
template <> __device__ __forceinline__ void cp_async<8>(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
template <> __device__ __forceinline__ void cp_async<4>(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Streaming (evict-first) stores, used where the data is not read again soon.
__device__ __forceinline__ void st_stream(uint4* p, uint4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint2* p, uint2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint32_t* p, uint32_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint16_t* p, uint16_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint8_t* p, uint8_t v) { __stcs(p, v); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar`, giving up after `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Wait until the 32-bit word at p satisfies `done(value)`, giving up after
// `limit` SM cycles; returns the last value read and sets *ok.  Every wait on
// a flag written by another CTA goes through here, so one limit (the
// context's) bounds them all.
template <class Done>
__device__ __forceinline__ uint32_t wait_word_bounded(const uint32_t* p, long long limit, bool* ok, Done done) {
  const volatile uint32_t* v = p;
  const long long t0 = clock64();
  uint32_t x = *v;
  while (!done(x)) {
    if (clock64() - t0 > limit) {
      *ok = false;
      return x;
    }
    __nanosleep(32);
    x = *v;
  }
  *ok = true;
  return x;
}

}  // namespace dpg
