// C ABI of the record-retrieval library (declarations and contracts in
// include/dpg.h): contexts, scratch memory, argument checks and the entry
// points that enqueue the kernels of dpg_retrieve.cu.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "dpg_device.cuh"
#include "dpg_internal.h"

namespace {

// Makes ctx->device current for the scope of an API call and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!na || !nb) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

constexpr uint64_t kMaxCount = 0x7fffffffULL;  // n and n_src fit in int32

// Shared checks of a retrieval request; `rid_bytes` is the byte span the rids
// occupy (for the overlap check).
int check_retrieval(const dpg_ctx* ctx, const void* src, size_t n_src, size_t rec, size_t n, const void* rids,
                    size_t rid_bytes, const void* dst) {
  if (!ctx || rec == 0) return DPG_EINVAL;
  if (n > kMaxCount || n_src > kMaxCount) return DPG_EINVAL;
  if (rec > (1ull << 30)) return DPG_EINVAL;
  if (n == 0) return DPG_OK;
  if (!rids || !dst || (n_src > 0 && !src)) return DPG_EINVAL;
  if (overlaps(src, n_src * rec, dst, n * rec)) return DPG_EINVAL;
  if (overlaps(rids, rid_bytes, dst, n * rec)) return DPG_EINVAL;
  return DPG_OK;
}

}  // namespace

namespace dpg {

int cuda_fail(dpg_ctx& ctx, cudaError_t e, const char* what) {
  ctx.last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return DPG_ECUDA;
}

TraceScope::TraceScope(dpg_ctx& c, const char* name, cudaStream_t s) : ctx(c), stream(s), on(c.trace) {
  if (!on) return;
  dpg_ctx::TraceRec r{name, nullptr, nullptr};
  for (cudaEvent_t* e : {&r.start, &r.stop}) {
    if (!ctx.trace_pool.empty()) {
      *e = ctx.trace_pool.back();
      ctx.trace_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      on = false;
      return;
    }
  }
  cudaEventRecord(r.start, stream);
  ctx.trace_pending.push_back(r);
}

TraceScope::~TraceScope() {
  if (on) cudaEventRecord(ctx.trace_pending.back().stop, stream);
}

// Folds finished trace records into the per-kernel totals.
static void trace_collect(dpg_ctx& ctx) {
  for (auto& r : ctx.trace_pending) {
    float ms = 0.f;
    cudaEventSynchronize(r.stop);
    cudaEventElapsedTime(&ms, r.start, r.stop);
    auto it = ctx.trace_totals.find(r.name);
    if (it == ctx.trace_totals.end()) {
      ctx.trace_names.push_back(r.name);
      it = ctx.trace_totals.emplace(r.name, std::make_pair(0.0, uint64_t(0))).first;
    }
    it->second.first += ms;
    it->second.second += 1;
    ctx.trace_pool.push_back(r.start);
    ctx.trace_pool.push_back(r.stop);
  }
  ctx.trace_pending.clear();
}

// An allocation the test hook dpg_inject_alloc_failure asked to fail.
static bool injected_failure(dpg_ctx& ctx) {
  if (ctx.fail_allocs <= 0) return false;
  ctx.fail_allocs--;
  ctx.last_error = "injected allocation failure";
  return true;
}

int ensure_scratch(dpg_ctx& ctx, size_t bytes) {
  if (bytes <= ctx.scratch_bytes) return DPG_OK;
  if (ctx.external_memory) {
    ctx.last_error = "lent scratch too small";
    return DPG_ENOMEM;
  }
  if (injected_failure(ctx)) return DPG_ENOMEM;
  const size_t grain = size_t(2) << 20;
  const size_t want = (bytes + grain - 1) / grain * grain;
  if (ctx.scratch) {
    cudaError_t e = cudaFree(ctx.scratch);  // synchronizes the device
    ctx.scratch = nullptr;
    ctx.scratch_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(scratch)");
  }
  cudaError_t e = cudaMalloc(&ctx.scratch, want);
  if (e != cudaSuccess) {
    ctx.scratch = nullptr;
    cudaGetLastError();
    ctx.last_error = std::string("cudaMalloc(scratch): ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DPG_ENOMEM : DPG_ECUDA;
  }
  ctx.scratch_bytes = want;
  return DPG_OK;
}

int ensure_aux(dpg_ctx& ctx, size_t bytes) {
  if (bytes <= ctx.aux_bytes) return DPG_OK;
  if (ctx.external_memory) {
    ctx.last_error = "lent work space too small";
    return DPG_ENOMEM;
  }
  if (injected_failure(ctx)) return DPG_ENOMEM;
  const size_t grain = size_t(2) << 20;
  const size_t want = (bytes + grain - 1) / grain * grain;
  if (ctx.aux) {
    cudaError_t e = cudaFree(ctx.aux);
    ctx.aux = nullptr;
    ctx.aux_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(aux)");
  }
  cudaError_t e = cudaMalloc(&ctx.aux, want);
  if (e != cudaSuccess) {
    ctx.aux = nullptr;
    cudaGetLastError();
    ctx.last_error = std::string("cudaMalloc(aux): ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DPG_ENOMEM : DPG_ECUDA;
  }
  ctx.aux_bytes = want;
  return DPG_OK;
}

}  // namespace dpg

extern "C" {

const char* dpg_strerror(dpg_status s) {
  switch (s) {
    case DPG_OK: return "ok";
    case DPG_EINVAL: return "invalid argument";
    case DPG_ERANGE: return "rid or key out of range";
    case DPG_ENOMEM: return "out of device memory";
    case DPG_ECUDA: return "CUDA runtime error";
    case DPG_ETIMEOUT: return "device-side wait timed out";
    case DPG_EBUSY: return "resource busy";
  }
  return "unknown status";
}

dpg_status dpg_ctx_create(dpg_ctx** out, int device) {
  if (!out) return DPG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DPG_EINVAL;
  }
  dpg_ctx* c = new (std::nothrow) dpg_ctx();
  if (!c) return DPG_ENOMEM;
  c->device = device;
  DeviceGuard g(device);
  int smem = 0;
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_khz, cudaDevAttrClockRate, device) != cudaSuccess ||
      cudaMalloc(&c->d_err, dpg::kErrBlockBytes) != cudaSuccess ||
      cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->d_err, 0, dpg::kErrBlockBytes) != cudaSuccess) {
    cudaGetLastError();
    if (c->d_err) cudaFree(c->d_err);
    if (c->h_err) cudaFreeHost(c->h_err);
    delete c;
    return DPG_ECUDA;
  }
  c->smem_optin = (size_t)smem;
  *out = c;
  return DPG_OK;
}

void dpg_ctx_destroy(dpg_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (auto& r : c->trace_pending) {
      cudaEventDestroy(r.start);
      cudaEventDestroy(r.stop);
    }
    for (cudaEvent_t e : c->trace_pool) cudaEventDestroy(e);
    if (c->io) cudaFree(c->io);
    if (c->aux && !c->external_memory) cudaFree(c->aux);
    if (c->batch_host) cudaFreeHost(c->batch_host);
    if (c->scratch && !c->external_memory) cudaFree(c->scratch);
    if (c->d_err) cudaFree(c->d_err);
    if (c->h_err) cudaFreeHost(c->h_err);
  }
  delete c;
}

const char* dpg_last_error(dpg_ctx* c) { return c ? c->last_error.c_str() : ""; }

dpg_status dpg_set_wait_limit(dpg_ctx* c, double seconds) {
  if (!c || !(seconds > 0.0) || seconds > 60.0) return DPG_EINVAL;
  const double khz = c->sm_khz > 0 ? (double)c->sm_khz : 2.07e6;
  c->wait_cycles = std::max<long long>(1, (long long)(seconds * khz * 1e3));
  return DPG_OK;
}

dpg_status dpg_check_wait(dpg_ctx* c, void* stream) {
  if (!c) return DPG_EINVAL;
  DeviceGuard g(c->device);
  const uint32_t* never = reinterpret_cast<const uint32_t*>(c->d_err) + dpg::kErrNeverSetWord;
  return (dpg_status)dpg::launch_wait_check(*c, never, static_cast<cudaStream_t>(stream));
}

dpg_status dpg_inject_alloc_failure(dpg_ctx* c, int count) {
  if (!c || count < 0) return DPG_EINVAL;
  c->fail_allocs = count;
  return DPG_OK;
}

uint64_t dpg_kernel_launches(dpg_ctx* c) { return c ? c->launches : 0; }

dpg_status dpg_retrieve(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t n, const int32_t* rids,
                        void* dst, void* stream) {
  int s = check_retrieval(c, src, n_src, rec, n, rids, n * 4, dst);
  if (s != DPG_OK || n == 0) return (dpg_status)s;
  if (rec > dpg::kMaxDpgRecBytes) return DPG_EINVAL;
  DeviceGuard g(c->device);
  dpg::Retrieval r{static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, n,
                   dpg::RidSpec{reinterpret_cast<const uint8_t*>(rids), 4}, static_cast<uint8_t*>(dst),
                   static_cast<cudaStream_t>(stream)};
  return (dpg_status)dpg::run_dpg(*c, r, dpg::choose_plan(*c, r));
}

dpg_status dpg_retrieve_direct(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t n,
                               const int32_t* rids, void* dst, void* stream) {
  int s = check_retrieval(c, src, n_src, rec, n, rids, n * 4, dst);
  if (s != DPG_OK || n == 0) return (dpg_status)s;
  DeviceGuard g(c->device);
  dpg::Retrieval r{static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, n,
                   dpg::RidSpec{reinterpret_cast<const uint8_t*>(rids), 4}, static_cast<uint8_t*>(dst),
                   static_cast<cudaStream_t>(stream)};
  return (dpg_status)dpg::run_direct(*c, r);
}

static int check_pairs(size_t stride, size_t rid_off) {
  if (stride < 4 || stride % 4 || rid_off % 4 || rid_off + 4 > stride || stride > (1u << 20)) return DPG_EINVAL;
  return DPG_OK;
}

dpg_status dpg_sort_copy(dpg_ctx* c, const void* pairs, size_t stride, size_t rid_off, size_t n, const void* src,
                         size_t n_src, size_t rec, void* dst, void* stream) {
  if (check_pairs(stride, rid_off)) return DPG_EINVAL;
  int s = check_retrieval(c, src, n_src, rec, n, pairs, n * stride, dst);
  if (s != DPG_OK || n == 0) return (dpg_status)s;
  if (rec > dpg::kMaxDpgRecBytes || reinterpret_cast<uintptr_t>(pairs) % 4) return DPG_EINVAL;
  DeviceGuard g(c->device);
  dpg::Retrieval r{static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, n,
                   dpg::RidSpec{static_cast<const uint8_t*>(pairs) + rid_off, (uint32_t)stride},
                   static_cast<uint8_t*>(dst), static_cast<cudaStream_t>(stream)};
  return (dpg_status)dpg::run_dpg(*c, r, dpg::choose_plan(*c, r));
}

dpg_status dpg_sort_copy_direct(dpg_ctx* c, const void* pairs, size_t stride, size_t rid_off, size_t n,
                                const void* src, size_t n_src, size_t rec, void* dst, void* stream) {
  if (check_pairs(stride, rid_off)) return DPG_EINVAL;
  int s = check_retrieval(c, src, n_src, rec, n, pairs, n * stride, dst);
  if (s != DPG_OK || n == 0) return (dpg_status)s;
  if (reinterpret_cast<uintptr_t>(pairs) % 4) return DPG_EINVAL;
  DeviceGuard g(c->device);
  dpg::Retrieval r{static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, n,
                   dpg::RidSpec{static_cast<const uint8_t*>(pairs) + rid_off, (uint32_t)stride},
                   static_cast<uint8_t*>(dst), static_cast<cudaStream_t>(stream)};
  return (dpg_status)dpg::run_direct(*c, r);
}

dpg_status dpg_sync(dpg_ctx* c, void* stream) {
  if (!c) return DPG_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return (dpg_status)dpg::cuda_fail(*c, e, "dpg_sync");
  const int bits = *c->h_err;
  if (bits & dpg::ERR_RANGE) return DPG_ERANGE;
  if (bits & dpg::ERR_TIMEOUT) return DPG_ETIMEOUT;
  return DPG_OK;
}

// ---- §3 sort: key-pointer pairs and the whole three-phase sort.

static int check_sort(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t key_bytes, const void* out) {
  if (!c || rec == 0 || key_bytes == 0 || key_bytes > 12 || key_bytes > rec) return DPG_EINVAL;
  if (n_src > 0x7fffffffULL || rec > (1ull << 30)) return DPG_EINVAL;
  if (n_src && (!src || !out)) return DPG_EINVAL;
  return DPG_OK;
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

dpg_status dpg_sort_keyptr(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t key_bytes, void* pairs,
                           void* stream) {
  int s = check_sort(c, src, n_src, rec, key_bytes, pairs);
  if (s != DPG_OK || n_src == 0) return (dpg_status)s;
  if (overlaps(src, n_src * rec, pairs, n_src * 16)) return DPG_EINVAL;
  DeviceGuard g(c->device);
  const size_t bt = al256(dpg::sort_keyptr_tmp_bytes(n_src, (uint32_t)key_bytes)), bs = dpg::sort_scan_bytes(n_src);
  if ((s = dpg::ensure_aux(*c, bt + bs))) return (dpg_status)s;
  uint8_t* tmp = static_cast<uint8_t*>(c->aux);
  return (dpg_status)dpg::run_sort_keyptr(*c, static_cast<const uint8_t*>(src), n_src, (uint32_t)rec,
                                          (uint32_t)key_bytes, static_cast<uint8_t*>(pairs), tmp, tmp + bt,
                                          static_cast<cudaStream_t>(stream));
}

dpg_status dpg_sort_records(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t key_bytes, void* dst,
                            void* stream) {
  int s = check_sort(c, src, n_src, rec, key_bytes, dst);
  if (s != DPG_OK || n_src == 0) return (dpg_status)s;
  if (rec > dpg::kMaxDpgRecBytes || overlaps(src, n_src * rec, dst, n_src * rec)) return DPG_EINVAL;
  DeviceGuard g(c->device);
  const size_t bp = al256(n_src * 16), bt = al256(dpg::sort_keyptr_tmp_bytes(n_src, (uint32_t)key_bytes)),
               bs = dpg::sort_scan_bytes(n_src);
  if ((s = dpg::ensure_aux(*c, bp + bt + bs))) return (dpg_status)s;
  uint8_t* pairs = static_cast<uint8_t*>(c->aux);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = dpg::run_sort_keyptr(*c, static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, (uint32_t)key_bytes, pairs,
                           pairs + bp, pairs + bp + bt, st);
  if (s != DPG_OK) return (dpg_status)s;
  dpg::Retrieval r{static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, n_src,
                   dpg::RidSpec{pairs + 12, 16}, static_cast<uint8_t*>(dst), st};
  return (dpg_status)dpg::run_dpg(*c, r, dpg::choose_plan(*c, r));
}

// ---- plan tuning

dpg_status dpg_tune(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t n, const void* rid_base,
                    size_t rid_stride, void* dst, void* stream, int* variant, int* seg_log2) {
  if (rid_stride < 4 || rid_stride % 4) return DPG_EINVAL;
  int s = check_retrieval(c, src, n_src, rec, n, rid_base, n * rid_stride, dst);
  if (s != DPG_OK) return (dpg_status)s;
  if (n == 0 || n_src == 0 || rec > dpg::kMaxDpgRecBytes || reinterpret_cast<uintptr_t>(rid_base) % 4)
    return n == 0 ? DPG_OK : DPG_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dpg::Retrieval r{static_cast<const uint8_t*>(src), n_src, (uint32_t)rec, n,
                   dpg::RidSpec{static_cast<const uint8_t*>(rid_base), (uint32_t)rid_stride},
                   static_cast<uint8_t*>(dst), st};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return DPG_ECUDA;
  }
  const bool was_tracing = c->trace;
  c->trace = false;
  float best = 1e30f;
  dpg::Plan best_plan;
  int rc = DPG_OK;
  for (const dpg::Plan& p : dpg::plan_candidates(*c, r)) {
    rc = dpg::run_dpg(*c, r, p);  // warm-up, sizes the scratch
    if (rc == DPG_OK) rc = dpg_sync(c, stream);
    if (rc != DPG_OK) break;
    float total = 0.f;
    for (int rep = 0; rep < 2 && rc == DPG_OK; ++rep) {
      cudaEventRecord(e0, st);
      rc = dpg::run_dpg(*c, r, p);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
    if (rc == DPG_OK) rc = dpg_sync(c, stream);
    if (rc != DPG_OK) break;
    if (total < best) {
      best = total;
      best_plan = p;
    }
  }
  c->trace = was_tracing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DPG_OK) return (dpg_status)rc;
  c->plans[dpg::plan_key(r)] = {best_plan.variant, best_plan.seg_log2};
  if (variant) *variant = best_plan.variant;
  if (seg_log2) *seg_log2 = best_plan.seg_log2;
  return DPG_OK;
}

void dpg_last_plan(dpg_ctx* c, int* variant, int* seg_log2) {
  if (!c) return;
  if (variant) *variant = c->last_variant;
  if (seg_log2) *seg_log2 = c->last_seg_log2;
}

void dpg_trace_enable(dpg_ctx* c, int on) {
  if (!c) return;
  DeviceGuard g(c->device);
  dpg::trace_collect(*c);
  c->trace = on != 0;
}

void dpg_trace_reset(dpg_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  dpg::trace_collect(*c);
  c->trace_totals.clear();
  c->trace_names.clear();
}

size_t dpg_trace_count(dpg_ctx* c) {
  if (!c) return 0;
  DeviceGuard g(c->device);
  dpg::trace_collect(*c);
  return c->trace_names.size();
}

dpg_status dpg_trace_get(dpg_ctx* c, size_t index, const char** name, double* total_ms, uint64_t* launches) {
  if (!c || !name || !total_ms || !launches) return DPG_EINVAL;
  DeviceGuard g(c->device);
  dpg::trace_collect(*c);
  if (index >= c->trace_names.size()) return DPG_EINVAL;
  const auto& t = c->trace_totals[c->trace_names[index]];
  *name = c->trace_names[index].c_str();
  *total_ms = t.first;
  *launches = t.second;
  return DPG_OK;
}

// ---- host-buffer entry points: copy in, run on the device, copy out.

static int ensure_io(dpg_ctx& c, size_t bytes) {
  if (bytes <= c.io_bytes) return DPG_OK;
  if (dpg::injected_failure(c)) return DPG_ENOMEM;
  if (c.io) {
    cudaFree(c.io);
    c.io = nullptr;
    c.io_bytes = 0;
  }
  const size_t grain = size_t(2) << 20;
  const size_t want = (bytes + grain - 1) / grain * grain;
  cudaError_t e = cudaMalloc(&c.io, want);
  if (e != cudaSuccess) {
    c.io = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DPG_ENOMEM : dpg::cuda_fail(c, e, "cudaMalloc(io)");
  }
  c.io_bytes = want;
  return DPG_OK;
}

dpg_status dpg_retrieve_host(dpg_ctx* c, const void* src, size_t n_src, size_t rec, size_t n,
                             const int32_t* rids, void* dst, void* stream) {
  int s = check_retrieval(c, src, n_src, rec, n, rids, n * 4, dst);
  if (s != DPG_OK || n == 0) return (dpg_status)s;
  if (rec > dpg::kMaxDpgRecBytes) return DPG_EINVAL;
  DeviceGuard g(c->device);
  const size_t bs = al256(n_src * rec), br = al256(n * 4), bd = al256(n * rec);
  if ((s = ensure_io(*c, bs + br + bd))) return (dpg_status)s;
  uint8_t* d_src = static_cast<uint8_t*>(c->io);
  uint8_t* d_rids = d_src + bs;
  uint8_t* d_dst = d_rids + br;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(d_src, src, n_src * rec, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rids, rids, n * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (dpg_status)dpg::cuda_fail(*c, e, "copy in");
  s = dpg_retrieve(c, d_src, n_src, rec, n, reinterpret_cast<const int32_t*>(d_rids), d_dst, stream);
  if (s != DPG_OK) return (dpg_status)s;
  if ((s = dpg_sync(c, stream)) != DPG_OK) return (dpg_status)s;
  e = cudaMemcpyAsync(dst, d_dst, n * rec, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DPG_OK : (dpg_status)dpg::cuda_fail(*c, e, "copy out");
}

dpg_status dpg_sort_copy_host(dpg_ctx* c, const void* pairs, size_t stride, size_t rid_off, size_t n,
                              const void* src, size_t n_src, size_t rec, void* dst, void* stream) {
  if (check_pairs(stride, rid_off)) return DPG_EINVAL;
  int s = check_retrieval(c, src, n_src, rec, n, pairs, n * stride, dst);
  if (s != DPG_OK || n == 0) return (dpg_status)s;
  if (rec > dpg::kMaxDpgRecBytes) return DPG_EINVAL;
  DeviceGuard g(c->device);
  const size_t bs = al256(n_src * rec), bp = al256(n * stride), bd = al256(n * rec);
  if ((s = ensure_io(*c, bs + bp + bd))) return (dpg_status)s;
  uint8_t* d_src = static_cast<uint8_t*>(c->io);
  uint8_t* d_pairs = d_src + bs;
  uint8_t* d_dst = d_pairs + bp;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(d_src, src, n_src * rec, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pairs, pairs, n * stride, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (dpg_status)dpg::cuda_fail(*c, e, "copy in");
  s = dpg_sort_copy(c, d_pairs, stride, rid_off, n, d_src, n_src, rec, d_dst, stream);
  if (s != DPG_OK) return (dpg_status)s;
  if ((s = dpg_sync(c, stream)) != DPG_OK) return (dpg_status)s;
  e = cudaMemcpyAsync(dst, d_dst, n * rec, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DPG_OK : (dpg_status)dpg::cuda_fail(*c, e, "copy out");
}

}  // extern "C"
