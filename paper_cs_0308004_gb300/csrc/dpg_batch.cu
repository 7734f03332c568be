// Batched record retrieval: many requests of uneven record counts and record
// sizes in one call (dpg_retrieve_batch in include/dpg.h).
//
// Requests that read the same source table with the same record size form a
// group, and a group is one DPG retrieval over the concatenation of its
// requests' rid lists: Phase II then probes each source segment once for the
// whole group instead of once per request.  A request's rids are checked
// against its own n_src while the group's rid list is assembled
// (k_batch_rids); destinations that are not laid out back to back are filled
// from a group staging buffer afterwards (k_batch_copy_out).  Everything is
// stream-ordered, so a warmed-up batch can be captured in a CUDA graph.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "dpg_device.cuh"
#include "dpg_internal.h"
#include "dpg_launch.cuh"

namespace dpg {
namespace {

struct BatchEntry {           // one request of a group, on the device
  const int32_t* rids;
  uint8_t* dst;
  uint64_t begin;             // first index of the request in the group's rid list
  uint64_t n;
  uint32_t n_src;
  uint32_t pad;
};

constexpr int kBatchThreads = 256;
constexpr uint64_t kBatchChunk = 8192;  // group indices per CTA step

// Request of group index g: the last entry with begin <= g, searched in [a, z].
__device__ __forceinline__ uint32_t entry_of(const BatchEntry* e, uint32_t a, uint32_t z, uint64_t g) {
  while (a < z) {
    const uint32_t m = (a + z + 1) >> 1;
    if (e[m].begin <= g) a = m;
    else z = m - 1;
  }
  return a;
}

// Assemble the group's rid list, checking each rid against its request's table size.
__global__ void __launch_bounds__(kBatchThreads)
    k_batch_rids(const BatchEntry* __restrict__ e, uint32_t ne, uint64_t total, int32_t* __restrict__ out,
                 int* err) {
  __shared__ uint32_t s_a, s_z;
  bool bad = false;
  for (uint64_t c0 = (uint64_t)blockIdx.x * kBatchChunk; c0 < total; c0 += (uint64_t)gridDim.x * kBatchChunk) {
    const uint64_t c1 = min(total, c0 + kBatchChunk);
    if (threadIdx.x == 0) {
      s_a = entry_of(e, 0, ne - 1, c0);
      s_z = entry_of(e, s_a, ne - 1, c1 - 1);
    }
    __syncthreads();
    const uint32_t a = s_a, z = s_z;
    for (uint64_t g = c0 + threadIdx.x; g < c1; g += kBatchThreads) {
      const uint32_t k = a == z ? a : entry_of(e, a, z, g);
      const int32_t r = __ldg(e[k].rids + (g - e[k].begin));
      if ((uint32_t)r >= e[k].n_src) {
        bad = true;
        out[g] = 0;
      } else {
        out[g] = r;
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(err, ERR_RANGE);
}

// Copy each request's slice of the group output (WB-byte words) to its dst.
template <int WB>
__global__ void __launch_bounds__(kBatchThreads)
    k_batch_copy_out(const BatchEntry* __restrict__ e, uint32_t ne, uint64_t total_rows, uint32_t W,
                     const uint8_t* __restrict__ tmp, const int* err) {
  using T = typename WordT<WB>::T;
  __shared__ uint32_t s_a, s_z;
  if (error_set(err)) return;
  const T* src = reinterpret_cast<const T*>(tmp);
  for (uint64_t c0 = (uint64_t)blockIdx.x * kBatchChunk; c0 < total_rows; c0 += (uint64_t)gridDim.x * kBatchChunk) {
    const uint64_t c1 = min(total_rows, c0 + kBatchChunk);
    if (threadIdx.x == 0) {
      s_a = entry_of(e, 0, ne - 1, c0);
      s_z = entry_of(e, s_a, ne - 1, c1 - 1);
    }
    __syncthreads();
    const uint32_t a = s_a, z = s_z;
    const uint64_t w0 = c0 * W, w1 = c1 * W;
    for (uint64_t t = w0 + threadIdx.x; t < w1; t += kBatchThreads) {
      const uint64_t g = t / W;
      const uint32_t k = a == z ? a : entry_of(e, a, z, g);
      reinterpret_cast<T*>(e[k].dst)[t - e[k].begin * W] = src[t];
    }
    __syncthreads();
  }
}

inline uint32_t align_of(uint64_t x) {
  uint32_t w = 16;
  while (w > 1 && (x % w)) w >>= 1;
  return w;
}

}  // namespace
}  // namespace dpg

extern "C" dpg_status dpg_retrieve_batch(dpg_ctx* c, const dpg_request* reqs, size_t count, void* stream) {
  using namespace dpg;
  if (!c || (count && !reqs)) return DPG_EINVAL;
  if (env_int("DPG_BATCH_GROUPED", 0) == 0) {
    // the persistent executor: every request a retrieval item
    std::vector<dpg_batch_item> items(count);
    for (size_t k = 0; k < count; ++k) {
      dpg_batch_item& it = items[k];
      std::memset(&it, 0, sizeof it);
      it.job.kind = DPG_JOB_RETRIEVE;
      it.job.src = reqs[k].src;
      it.job.n_src = reqs[k].n_src;
      it.job.rec_bytes = reqs[k].rec_bytes;
      it.job.n = reqs[k].n;
      it.job.rids = reqs[k].rids;
      it.out = reqs[k].dst;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    const int s = run_exec_batch(*c, items.data(), count, static_cast<cudaStream_t>(stream));
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return (dpg_status)s;
  }
  // host-side checks of every request, before anything is enqueued
  std::vector<size_t> live;
  for (size_t k = 0; k < count; ++k) {
    const dpg_request& q = reqs[k];
    if (q.rec_bytes == 0 || q.rec_bytes > kMaxDpgRecBytes || q.n > 0x7fffffffULL || q.n_src > 0x7fffffffULL)
      return DPG_EINVAL;
    if (q.n == 0) continue;
    if (!q.rids || !q.dst || (q.n_src && !q.src)) return DPG_EINVAL;
    live.push_back(k);
  }
  if (live.empty()) return DPG_OK;
  std::stable_sort(live.begin(), live.end(), [&](size_t x, size_t y) {
    const uintptr_t sx = reinterpret_cast<uintptr_t>(reqs[x].src), sy = reinterpret_cast<uintptr_t>(reqs[y].src);
    if (sx != sy) return sx < sy;
    return reqs[x].rec_bytes < reqs[y].rec_bytes;
  });
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  struct Restore {
    int d, cur;
    ~Restore() {
      if (d >= 0 && d != cur) cudaSetDevice(d);
    }
  } restore{prev, c->device};
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // groups and their device tables
  struct Group {
    size_t first, last;  // range in `live`
    uint64_t total;
    uint64_t n_src;
    bool rids_in_place, dst_in_place;
  };
  std::vector<Group> groups;
  for (size_t i = 0; i < live.size();) {
    size_t j = i;
    const dpg_request& q0 = reqs[live[i]];
    Group g{i, i, 0, 0, true, true};
    while (j < live.size() && reqs[live[j]].src == q0.src && reqs[live[j]].rec_bytes == q0.rec_bytes) {
      const dpg_request& q = reqs[live[j]];
      const uint64_t at = g.total;
      if (q.rids != q0.rids + at) g.rids_in_place = false;
      if (static_cast<uint8_t*>(q.dst) != static_cast<uint8_t*>(q0.dst) + at * q0.rec_bytes) g.dst_in_place = false;
      if (q.n_src != q0.n_src) g.rids_in_place = false;  // per-request range checks needed
      g.n_src = std::max<uint64_t>(g.n_src, q.n_src);
      g.total += q.n;
      ++j;
    }
    g.last = j;
    if (g.total > 0x7fffffffULL) return DPG_EINVAL;
    groups.push_back(g);
    i = j;
  }
  // one device table of BatchEntry for all groups, staged through pinned host memory
  const size_t n_entries = live.size();
  const size_t table_bytes = (n_entries * sizeof(BatchEntry) + 255) & ~size_t(255);
  size_t aux_need = table_bytes;
  for (const Group& g : groups) {
    const size_t rec = reqs[live[g.first]].rec_bytes;
    size_t need = table_bytes;
    if (!g.rids_in_place) need += (g.total * 4 + 255) & ~size_t(255);
    if (!g.dst_in_place) need += (g.total * rec + 255) & ~size_t(255);
    aux_need = std::max(aux_need, need);
  }
  if (int s = ensure_aux(*c, aux_need)) return (dpg_status)s;
  if (c->batch_host_bytes < table_bytes) {
    if (c->batch_host) cudaFreeHost(c->batch_host);
    c->batch_host = nullptr;
    c->batch_host_bytes = 0;
    if (cudaMallocHost(&c->batch_host, table_bytes) != cudaSuccess) {
      cudaGetLastError();
      return DPG_ENOMEM;
    }
    c->batch_host_bytes = table_bytes;
  }
  BatchEntry* host = static_cast<BatchEntry*>(c->batch_host);
  for (const Group& g : groups) {
    uint64_t at = 0;
    for (size_t i = g.first; i < g.last; ++i) {
      const dpg_request& q = reqs[live[i]];
      host[i] = BatchEntry{q.rids, static_cast<uint8_t*>(q.dst), at, q.n, (uint32_t)q.n_src, 0u};
      at += q.n;
    }
  }
  BatchEntry* dev_table = static_cast<BatchEntry*>(c->aux);
  cudaError_t e = cudaMemcpyAsync(dev_table, host, n_entries * sizeof(BatchEntry), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (dpg_status)cuda_fail(*c, e, "batch table");
  uint8_t* work = static_cast<uint8_t*>(c->aux) + table_bytes;

  for (const Group& g : groups) {
    const dpg_request& q0 = reqs[live[g.first]];
    const uint32_t rec = (uint32_t)q0.rec_bytes;
    const uint32_t ne = (uint32_t)(g.last - g.first);
    const BatchEntry* te = dev_table + g.first;
    const int32_t* rids = q0.rids;
    uint8_t* p = work;
    if (!g.rids_in_place) {
      int32_t* cat = reinterpret_cast<int32_t*>(p);
      p += (g.total * 4 + 255) & ~size_t(255);
      const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((g.total + kBatchChunk - 1) / kBatchChunk,
                                                                    (uint64_t)c->sms * 4));
      TraceScope ts(*c, "k_batch_rids", st);
      k_batch_rids<<<grid, kBatchThreads, 0, st>>>(te, ne, g.total, cat, c->d_err);
      c->launches++;
      rids = cat;
    }
    uint8_t* dst = g.dst_in_place ? static_cast<uint8_t*>(q0.dst) : p;
    Retrieval r{static_cast<const uint8_t*>(q0.src), g.n_src, rec, g.total,
                RidSpec{reinterpret_cast<const uint8_t*>(rids), 4}, dst, st};
    if (int s = run_dpg(*c, r, choose_plan(*c, r))) return (dpg_status)s;
    if (!g.dst_in_place) {
      uint32_t wb = align_of(rec);
      for (size_t i = g.first; i < g.last; ++i)
        wb = std::min(wb, align_of(reinterpret_cast<uintptr_t>(reqs[live[i]].dst)));
      const uint32_t W = rec / wb;
      const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((g.total + kBatchChunk - 1) / kBatchChunk,
                                                                    (uint64_t)c->sms * 4));
      TraceScope ts(*c, "k_batch_copy_out", st);
      switch (wb) {
        case 16: k_batch_copy_out<16><<<grid, kBatchThreads, 0, st>>>(te, ne, g.total, W, dst, c->d_err); break;
        case 8: k_batch_copy_out<8><<<grid, kBatchThreads, 0, st>>>(te, ne, g.total, W, dst, c->d_err); break;
        case 4: k_batch_copy_out<4><<<grid, kBatchThreads, 0, st>>>(te, ne, g.total, W, dst, c->d_err); break;
        case 2: k_batch_copy_out<2><<<grid, kBatchThreads, 0, st>>>(te, ne, g.total, W, dst, c->d_err); break;
        default: k_batch_copy_out<1><<<grid, kBatchThreads, 0, st>>>(te, ne, g.total, W, dst, c->d_err); break;
      }
      c->launches++;
    }
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? DPG_OK : (dpg_status)cuda_fail(*c, e, "batch launch");
}
