// Foreign-key joins with DPG (§4.2.1) on sm_103a.
//
// The fact relation (R in §4.2) carries an int32 foreign key per row; the
// dimension relation (F) is indexed by its int64 key, which here equals its
// row number, so the join triple of fact row i is (k, rid_R = i, rid_F = fk_i)
// (§4.2.2) and needs no index lookup.  Output rows are fact row || dimension
// row.
//
//   DPG-move: move F's rows into R's order by DPG retrieval with the fk column
//             as the rid sequence; Phase III writes fact[i] || dim[fk_i].
//   DPG-sort: sort the rid pairs (rid_F, rid_R) by rid_F (stable radix sort of
//             8-byte pairs on the low bytes of fk), then move R's rows into that order by DPG
//             retrieval; Phase III writes fact row || dim[fk].
//   direct:   out[i] = fact[i] || dim[fk_i] in one pass (baseline).
#include <algorithm>

#include "dpg_device.cuh"
#include "dpg_internal.h"

namespace dpg {
namespace {

// Pair i of the DPG-sort join (8 bytes): key bytes [0, kb) = fk big-endian
// in the first word, rid = i in the second; the digit counts of each key
// byte are taken on the way (counts[j * 256 + d], zero on entry).  A
// foreign key outside [0, n_dim) raises the range bit.
__global__ void __launch_bounds__(256)
    k_extract_fk_pairs(const uint8_t* __restrict__ fact, uint64_t n, uint32_t fact_bytes, uint32_t fk_off,
                       uint64_t n_dim, uint32_t kb, uint2* __restrict__ pairs, uint32_t* __restrict__ counts,
                       int* err) {
  __shared__ uint32_t h[4 * 256];
  for (uint32_t x = threadIdx.x; x < kb * 256; x += blockDim.x) h[x] = 0;
  __syncthreads();
  bool bad = false;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t fk = (uint32_t)__ldg(reinterpret_cast<const int32_t*>(fact + i * fact_bytes + fk_off));
    if ((uint64_t)fk >= n_dim) bad = true;
    uint32_t key = 0;
    for (uint32_t j = 0; j < kb; ++j) key |= ((fk >> (8 * (kb - 1 - j))) & 0xffu) << (8 * j);
    pairs[i] = make_uint2(key, (uint32_t)i);
    for (uint32_t j = 0; j < kb; ++j) atomicAdd(&h[j * 256 + ((key >> (8 * j)) & 0xffu)], 1u);
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < kb * 256; x += blockDim.x)
    if (h[x]) atomicAdd(&counts[x], h[x]);
  if (bad) atomicOr(err, ERR_RANGE);
}

}  // namespace
}  // namespace dpg

namespace {

bool overlaps2(const void* a, size_t na, const void* b, size_t nb) {
  if (!na || !nb) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" dpg_status dpg_fk_join(dpg_ctx* c, const void* fact_v, size_t n_fact, size_t fact_bytes, size_t fk_off,
                                  const void* dim_v, size_t n_dim, size_t dim_bytes, size_t pk_off, void* out_v,
                                  int mode, void* stream) {
  using namespace dpg;
  if (!c || mode < 0 || mode > 2) return DPG_EINVAL;
  if (fact_bytes < 4 || fact_bytes % 4 || fk_off % 4 || fk_off + 4 > fact_bytes) return DPG_EINVAL;
  if (dim_bytes < 8 || pk_off + 8 > dim_bytes) return DPG_EINVAL;
  if (n_fact > 0x7fffffffULL || n_dim > 0x7fffffffULL || fact_bytes > kMaxDpgRecBytes ||
      dim_bytes > kMaxDpgRecBytes)
    return DPG_EINVAL;
  // join rows are walked as word indices t < n_fact * row_w divided by the
  // row's word count row_w (at most (fact_bytes + dim_bytes) one-byte words):
  // the multiply-high division is exact only while t * row_w < 2^64
  if (!fastdiv_exact((uint32_t)(fact_bytes + dim_bytes), (uint64_t)n_fact * (fact_bytes + dim_bytes)))
    return DPG_EINVAL;
  if (n_fact == 0) return DPG_OK;
  if (!fact_v || !out_v || (n_dim && !dim_v) || reinterpret_cast<uintptr_t>(fact_v) % 4) return DPG_EINVAL;
  const size_t out_bytes = n_fact * (fact_bytes + dim_bytes);
  if (overlaps2(fact_v, n_fact * fact_bytes, out_v, out_bytes) || overlaps2(dim_v, n_dim * dim_bytes, out_v, out_bytes))
    return DPG_EINVAL;
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != c->device) cudaSetDevice(c->device);
  struct Restore {
    int d, cur;
    ~Restore() {
      if (d >= 0 && d != cur) cudaSetDevice(d);
    }
  } restore{dev_prev, c->device};

  const uint8_t* fact = static_cast<const uint8_t*>(fact_v);
  const uint8_t* dim = static_cast<const uint8_t*>(dim_v);
  uint8_t* out = static_cast<uint8_t*>(out_v);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  JoinSpec j{mode == 2 ? 0 : mode, fact, (uint32_t)fact_bytes, (uint32_t)fk_off, dim, (uint32_t)dim_bytes,
             (uint32_t)pk_off, n_dim, out, nullptr, 0};

  if (mode == 2) return (dpg_status)run_join_direct(*c, j, n_fact, st);

  if (mode == 0) {
    Retrieval r{dim, n_dim, (uint32_t)dim_bytes, n_fact, RidSpec{fact + fk_off, (uint32_t)fact_bytes}, out, st};
    r.join = &j;
    return (dpg_status)run_dpg(*c, r, choose_plan(*c, r));
  }

  // DPG-sort: stable sort of (fk, i) on the bytes fk can occupy, then move
  // the fact rows into that order.
  uint32_t kb = 1;
  while (kb < 4 && n_dim > (1ull << (8 * kb))) ++kb;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t bp = al(n_fact * 8), bs = sort_scan_bytes(n_fact);
  if (int s = ensure_aux(*c, 2 * bp + bs)) return (dpg_status)s;
  uint8_t* a = static_cast<uint8_t*>(c->aux);
  uint32_t* counts = radix_counts(a + 2 * bp);
  if (cudaError_t e = cudaMemsetAsync(counts, 0, 12 * 256 * 4, st)) return (dpg_status)cuda_fail(*c, e, "memset");
  {
    TraceScope ts(*c, "k_extract_fk_pairs", st);
    const int grid = (int)std::min<uint64_t>((n_fact + 255) / 256, (uint64_t)c->sms * 8);
    k_extract_fk_pairs<<<grid, 256, 0, st>>>(fact, n_fact, (uint32_t)fact_bytes, (uint32_t)fk_off, n_dim, kb,
                                             reinterpret_cast<uint2*>(a), counts, c->d_err);
    c->launches++;
  }
  int status = DPG_OK;
  uint8_t* sorted = run_radix_pairs8(*c, a, a + bp, a + 2 * bp, n_fact, kb, st, &status);
  if (status != DPG_OK) return (dpg_status)status;
  j.sorted_pairs = sorted;
  j.key_bytes = kb;
  Retrieval r{fact, n_fact, (uint32_t)fact_bytes, n_fact, RidSpec{sorted + 4, 8}, out, st};
  r.join = &j;
  return (dpg_status)run_dpg(*c, r, choose_plan(*c, r));
}
