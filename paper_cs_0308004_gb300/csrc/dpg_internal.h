// Host-side internals of the record-retrieval library: the context object,
// plans and the launch functions behind the C ABI in include/dpg.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dpg.h"

struct dpg_ctx {
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;     // max dynamic shared memory per block (opt-in)
  int* d_err = nullptr;      // device error word (bits dpg::ERR_*)
  long long wait_cycles = 2000000000LL;  // limit of device waits on other CTAs' flags (SM cycles)
  int sm_khz = 0;            // SM clock rate, to turn dpg_set_wait_limit's time into cycles
  int fail_allocs = 0;       // allocations left to fail (dpg_inject_alloc_failure)
  int* h_err = nullptr;      // pinned host copy used by dpg_sync
  void* scratch = nullptr;   // grown on demand
  size_t scratch_bytes = 0;
  bool external_memory = false;  // scratch and aux lent by a server: never grown or freed here
  uint64_t launches = 0;
  std::string last_error;
  // host-buffer entry points: device copies of the caller's tables
  void* io = nullptr;
  size_t io_bytes = 0;
  // sort and join work space (kept apart from the retrieval scratch, which a
  // sort or join hands to a retrieval while its own buffers are live)
  void* aux = nullptr;
  size_t aux_bytes = 0;
  // pinned staging of batch request tables (read again when a captured batch
  // graph replays)
  void* batch_host = nullptr;
  size_t batch_host_bytes = 0;
  // kernel tracing: CUDA events recorded around every launch on its stream
  bool trace = false;
  struct TraceRec {
    const char* name;
    cudaEvent_t start, stop;
  };
  std::vector<TraceRec> trace_pending;
  std::vector<cudaEvent_t> trace_pool;
  std::map<std::string, std::pair<double, uint64_t>> trace_totals;  // name -> (ms, launches)
  std::vector<std::string> trace_names;                              // stable order for readers
  // plans chosen by dpg_tune, keyed by retrieval shape, and the last plan run
  std::map<uint64_t, std::pair<int, int>> plans;  // key -> (variant, seg_log2)
  int last_variant = 0, last_seg_log2 = 0;
};

namespace dpg {

// How a retrieval is carried out.
//   variant 4: runs of a few MB held in the L2 (dpg_runs.cu): Phase I tile
//              counting sort into at most kL2MaxRuns runs -> Phase II gather in
//              run order -> Phase III tile rebuild or slot gather.
//   variant 3: runs (segments) held in shared memory: Phase I distribute ->
//              Phase II probe into an INTERNAL staging table in run order ->
//              Phase III gather in rid order (Figure 1).
//   variant 2: as variant 3, Phase II writing each record straight to its
//              destination slot (probe and gather fused).
struct Plan {
  int variant = 3;
  int seg_log2 = 10;     // a source segment (run) holds 2^seg_log2 records
  uint32_t chunk = 0;    // max rids per probe work item (0: 4 x segment)
};

// Where the rids come from: a plain int32 array, or the int32 field at a fixed
// offset of strided key-pointer pairs.
struct RidSpec {
  const uint8_t* base;   // address of rid 0
  uint32_t stride;       // bytes between consecutive rids (4 for a plain array)
};

// A foreign-key join riding on a retrieval (§4.2.1): Phase III writes join
// rows instead of plain records.
//   mode 0 (DPG-move): the retrieval moves dimension rows into fact order;
//          out row i = fact[i] || INTERNAL[slot[i]].  Phase II checks that
//          each probed dimension row's key equals its row number.
//   mode 1 (DPG-sort): the retrieval moves fact rows into the order of the
//          8-byte (fk, fact row) pairs sorted by fk; out row j = fact row j
//          of that order || dim[fk_j], the key of dim[fk_j] checked as it is
//          copied.  On the L2-run plan (fact rows up to 128 bytes) Phase III
//          rebuilds tiles of fact rows and reads fk_j from the staged row;
//          otherwise it reads INTERNAL[slot[j]] and decodes fk_j from sorted
//          pair j (key bytes [0, key_bytes) hold fk big-endian).
struct JoinSpec {
  int mode;
  const uint8_t* fact;
  uint32_t fact_bytes;
  uint32_t fk_off;
  const uint8_t* dim;
  uint32_t dim_bytes;
  uint32_t pk_off;
  uint64_t n_dim;
  uint8_t* out;
  const uint8_t* sorted_pairs;
  uint32_t key_bytes;
};

struct Retrieval {
  const uint8_t* src;
  uint64_t n_src;
  uint32_t rec;
  uint64_t n;
  RidSpec rids;
  uint8_t* dst;
  cudaStream_t stream;
  const JoinSpec* join = nullptr;
};

// The context's device error block: word 0 is the error word (bits
// dpg::ERR_*); word kErrNeverSetWord, on a line of its own, stays zero for
// ever (the flag dpg_check_wait waits on).
constexpr size_t kErrBlockBytes = 256;
constexpr size_t kErrNeverSetWord = 32;

// One kernel waiting, under ctx.wait_cycles, for *flag to become non-zero
// (dpg_check_wait; dpg_retrieve.cu).
int launch_wait_check(dpg_ctx& ctx, const uint32_t* flag, cudaStream_t st);

// Limits of the DPG path.
constexpr uint32_t kMaxDpgRecBytes = 65536;   // a segment holds at least one record
constexpr uint32_t kSmemBuckets = 24576;      // Phase I per-CTA counters fit in 96 KB
constexpr uint32_t kL2MaxRuns = 1024;         // runs of the L2-run plan (variant 4)

// Plan chosen for a retrieval: environment overrides (DPG_VARIANT,
// DPG_SEG_LOG2, DPG_CHUNK, DPG_L2_RUN_KB; DPG_L2_SLOT and
// DPG_UNPART_STAGE_MAX pick the L2-run plan's Phase III, DPG_GATHER_CTAS the
// grid of the grid-stride gathers) when set, else a plan dpg_tune
// cached for the retrieval's shape, else the default for its record size.
Plan choose_plan(const dpg_ctx& ctx, const Retrieval& r);
uint64_t plan_key(const Retrieval& r);
// Candidate plans the tuner times for a retrieval.
std::vector<Plan> plan_candidates(const dpg_ctx& ctx, const Retrieval& r);

// Bytes of context scratch a retrieval will take (its plan as chosen now).
size_t retrieve_scratch_need(const dpg_ctx& ctx, const Retrieval& r);

// Enqueue the DPG retrieval / the direct gather.  Return a dpg_status.
int run_dpg(dpg_ctx& ctx, const Retrieval& r, const Plan& plan);
int run_direct(dpg_ctx& ctx, const Retrieval& r);

// The L2-run plan (variant 4, dpg_runs.cu) and its scratch bytes.
int run_dpg_l2(dpg_ctx& ctx, const Retrieval& r, const Plan& plan);
size_t l2_scratch_need(const dpg_ctx& ctx, const Retrieval& r, const Plan& plan, bool strided);

// dst[k] = src[slot[k]] for k in [0, n) by the grid-stride gather, in words of
// wb bytes (dpg_retrieve.cu); `name` labels the launch in traces.
void launch_slot_gather(dpg_ctx& ctx, uint32_t wb, const uint8_t* src, uint8_t* dst, const uint32_t* slot,
                        uint64_t n, uint32_t rec, uint32_t n_src, cudaStream_t st, const char* name);

// Phase III of a join riding on a retrieval (r.join set): join rows from the
// fact and dimension tables and INTERNAL (`stage`) read through `slot`
// (dpg_retrieve.cu).
void launch_join_phase3(dpg_ctx& ctx, const Retrieval& r, const uint8_t* stage, const uint32_t* slot);

// The batch executor (dpg_exec.cu): every item of a batch as one persistent
// kernel; the grouped multi-kernel batch (dpg_batch.cu) runs instead when
// DPG_BATCH_GROUPED=1.
int run_exec_batch(dpg_ctx& ctx, const dpg_batch_item* items, size_t count, cudaStream_t st);

// Scratch arena helpers (dpg_api.cu).
int ensure_scratch(dpg_ctx& ctx, size_t bytes);
int ensure_aux(dpg_ctx& ctx, size_t bytes);

// Foreign-key join output without DPG: out row i = fact[i] || dim[fk_i]
// (dpg_retrieve.cu), the baseline of the join modes.
int run_join_direct(dpg_ctx& ctx, const JoinSpec& j, uint64_t n_fact, cudaStream_t st);

// Stable LSD radix sort of 16-byte pairs on key bytes [0, key_bytes) (dpg_sort.cu).
// `a` holds the pairs; the result ends in `a` (even key_bytes) or `b`; the
// returned pointer says which.  run_radix_pairs8: the same for 8-byte pairs
// (key bytes [0, key_bytes <= 4) in the first word, the rid in the second).
// The caller fills radix_counts(scan) while it builds the pairs: the count
// of digit d of key byte j over all pairs at [j * 256 + d] (zeroed first).
uint32_t* radix_counts(uint8_t* scan);
uint8_t* run_radix_pairs(dpg_ctx& ctx, uint8_t* a, uint8_t* b, uint8_t* scan, uint64_t n, uint32_t key_bytes,
                         cudaStream_t st, int* status);
uint8_t* run_radix_pairs8(dpg_ctx& ctx, uint8_t* a, uint8_t* b, uint8_t* scan, uint64_t n, uint32_t key_bytes,
                          cudaStream_t st, int* status);

// Phases 1-2 of the §3 sort (dpg_sort.cu): sorted 16-byte key-pointer pairs;
// tmp holds sort_keyptr_tmp_bytes(n, key_bytes), scan sort_scan_bytes(n).
size_t sort_keyptr_tmp_bytes(uint64_t n, uint32_t key_bytes);
size_t sort_scan_bytes(uint64_t n);
int run_sort_keyptr(dpg_ctx& ctx, const uint8_t* src, uint64_t n, uint32_t rec, uint32_t key_bytes, uint8_t* pairs,
                    uint8_t* tmp, uint8_t* scan, cudaStream_t st);
int cuda_fail(dpg_ctx& ctx, cudaError_t e, const char* what);

// Brackets one kernel launch with CUDA events on its stream when tracing is on.
struct TraceScope {
  dpg_ctx& ctx;
  cudaStream_t stream;
  bool on;
  TraceScope(dpg_ctx& c, const char* name, cudaStream_t s);
  ~TraceScope();
};

}  // namespace dpg
