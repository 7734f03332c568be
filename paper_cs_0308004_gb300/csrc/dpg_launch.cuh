// Host-side launch helpers shared by the library's .cu files.
#pragma once

#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>
#include <utility>

#include <cuda_runtime.h>

namespace dpg {

// Largest power of two up to 16 that divides x (an address or a size): the
// widest word a kernel may move through it.
inline uint32_t pow2_align(uint64_t x) {
  uint32_t w = 16;
  while (w > 1 && (x % w)) w >>= 1;
  return w;
}

template <class K>
inline void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// CTAs of `kernel` resident on one SM at `threads` threads and `smem` bytes of
// dynamic shared memory (looked up once per kernel and size).
template <class K>
inline int resident_per_sm(K kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> cache;
  const std::pair<const void*, size_t> key{reinterpret_cast<const void*>(kernel), smem * 4096 + (size_t)threads};
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nblk = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, kernel, threads, smem) != cudaSuccess || nblk < 1) {
    cudaGetLastError();
    nblk = 1;
  }
  cache[key] = nblk;
  return nblk;
}

inline int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return (v && *v) ? std::atoi(v) : dflt;
}

}  // namespace dpg
