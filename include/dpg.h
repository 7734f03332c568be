/*
 * dpg.h — C ABI of the GB300 (sm_103a) record-retrieval library.
 *
 * Record retrieval (Cooperman, Ma, Nguyen, "DPG: A Cache-Efficient Accelerator
 * for Sorting and for Join Operators", §1 and §2): given a source table of
 * fixed-size records, a sequence of record ids (rids) and a destination
 * table, copy record rids[i] of the source into slot i of the destination:
 *
 *     for each i:  dst[i] = src[rids[i]]
 *
 * The library computes it with distribute-probe-gather (DPG, §2.1, Figure 1)
 * as CUDA kernels, and offers the plain one-pass gather as a baseline, the
 * copy phase of a key-pointer sort (§3) and the DPG-move / DPG-sort
 * foreign-key joins (§4.2.1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Tables are packed arrays of records: record k of a table of `rec_bytes`
 *    records starts at byte k * rec_bytes.  No padding, any alignment (wider
 *    vector paths are taken when pointers and sizes allow).
 *  - Pointers are DEVICE pointers owned by the caller unless a call says
 *    otherwise.  The library never frees them and keeps no reference after
 *    the call's GPU work has finished.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls are stream-ordered: they enqueue kernels and return.
 *  - Argument errors (DPG_EINVAL) are detected on the host, before anything is
 *    enqueued.  A rid (or foreign key) outside its table is detected on the
 *    GPU before any destination byte is written: the destination is left
 *    untouched and the NEXT dpg_sync on that context returns DPG_ERANGE.
 *  - A context owns scratch memory, grown on demand with cudaMalloc; growth
 *    synchronizes the device, so the first call at a given size should come
 *    before any CUDA-graph capture.  One context serves one stream at a time:
 *    calls on one context from several streams at once race on its scratch.
 *  - Sizes: record counts and rid values fit in int32 (n, n_src <= 2^31 - 1).
 */
#ifndef DPG_H
#define DPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DPG_OK = 0,
  DPG_EINVAL = 1,    /* bad argument: null pointer, zero record size, overlap, size limit */
  DPG_ERANGE = 2,    /* a rid / foreign key outside [0, n_src) (reported by dpg_sync) */
  DPG_ENOMEM = 3,    /* scratch allocation failed */
  DPG_ECUDA = 4,     /* a CUDA runtime call failed */
  DPG_ETIMEOUT = 5,  /* a bounded device-side wait gave up (reported by dpg_sync) */
  DPG_EBUSY = 6      /* resource held by another request (serving admission) */
} dpg_status;

typedef struct dpg_ctx dpg_ctx;

/* Create a context on CUDA device `device` (it becomes current for the call).
 * *out receives the handle. */
dpg_status dpg_ctx_create(dpg_ctx** out, int device);

/* Destroy a context: synchronizes its device and frees its scratch.  NULL is a no-op. */
void dpg_ctx_destroy(dpg_ctx* ctx);

/* A static, human-readable string for a status code. */
const char* dpg_strerror(dpg_status status);

/* Last CUDA error string recorded by the context (for DPG_ECUDA), or "". */
const char* dpg_last_error(dpg_ctx* ctx);

/*
 * Record retrieval by distribute-probe-gather (§2.1, Figure 1).
 *   src       n_src records of rec_bytes bytes (the INPUT file of §2.1)
 *   rids      n int32 record ids, each in [0, n_src) (RID_LIST)
 *   dst       n records of rec_bytes bytes (OUTPUT); must not overlap src
 * Phase I partitions the rids by source run (2^k consecutive records), Phase
 * II copies each run's records out in run order while the run sits in fast
 * memory, Phase III writes the destination in rid order.  n == 0 is a no-op.
 * Duplicated and skewed rids are allowed (§2, §2.3).  The plan is the one
 * dpg_tune cached for this shape, else chosen by record size: below 192 bytes
 * runs of about 16 MB held in the L2 (tile counting sort in Phase I; Phase III
 * rebuilds the destination tile by tile below 96 bytes, through a 4-byte slot
 * per rid from 96 bytes); from 192 bytes runs of up to 104 KB held in one
 * CTA's shared memory, records written straight to their destination (2-pass).
 */
dpg_status dpg_retrieve(dpg_ctx* ctx, const void* src, size_t n_src, size_t rec_bytes,
                        size_t n, const int32_t* rids, void* dst, void* stream);

/* The same result by the plain one-pass gather (§1, "standard approach"):
 * every destination record is read straight from its random source location.
 * Baseline for comparison.  On a bad rid the destination is left partly
 * written (slots with valid rids are copied) and dpg_sync returns DPG_ERANGE. */
dpg_status dpg_retrieve_direct(dpg_ctx* ctx, const void* src, size_t n_src, size_t rec_bytes,
                               size_t n, const int32_t* rids, void* dst, void* stream);

/*
 * Copy phase of a three-phase key-pointer sort (§3, phase 3): `pairs` holds n
 * sorted key-pointer pairs of pair_stride bytes whose int32 rid sits at byte
 * rid_off (pair_stride and rid_off multiples of 4; the library's own pair
 * layout is 16 bytes with the rid at byte 12).  dst[i] = src[rid of pairs[i]],
 * by distribute-probe-gather.
 */
dpg_status dpg_sort_copy(dpg_ctx* ctx, const void* pairs, size_t pair_stride, size_t rid_off,
                         size_t n, const void* src, size_t n_src, size_t rec_bytes, void* dst,
                         void* stream);

/* Plain one-pass gather for the sort copy phase (baseline). */
dpg_status dpg_sort_copy_direct(dpg_ctx* ctx, const void* pairs, size_t pair_stride,
                                size_t rid_off, size_t n, const void* src, size_t n_src,
                                size_t rec_bytes, void* dst, void* stream);

/*
 * Phases 1 and 2 of the three-phase sort (§3): the key-pointer pair of every
 * record (its first key_bytes bytes, 1 <= key_bytes <= 12, as the key), sorted
 * by key as unsigned byte strings, equal keys in rid order.  `pairs` receives
 * n_src pairs of 16 bytes: key bytes, zero padding to byte 12, int32 rid at
 * byte 12 (the layout dpg_sort_copy reads with pair_stride 16, rid_off 12).
 * Stable LSD radix passes on key bytes 1 and 0 (one byte per pass), then each
 * bucket of equal two-byte prefix sorted on the rest of the key and the rid;
 * buckets of more than 256 pairs (ties, skewed keys) go through the full LSD
 * sort in one cooperative launch.  Context scratch: about 32 bytes per record.
 */
dpg_status dpg_sort_keyptr(dpg_ctx* ctx, const void* src, size_t n_src, size_t rec_bytes, size_t key_bytes,
                           void* pairs, void* stream);

/* The whole §3 sort: dst[i] = the record of rank i in (key, rid) order, i.e.
 * dpg_sort_keyptr followed by dpg_sort_copy (DPG record retrieval).  Context
 * scratch: about 48 bytes per record. */
dpg_status dpg_sort_records(dpg_ctx* ctx, const void* src, size_t n_src, size_t rec_bytes, size_t key_bytes,
                            void* dst, void* stream);

/*
 * Foreign-key join (§4.2): the fact relation has n_fact rows of fact_bytes
 * bytes with an int32 foreign key at byte fk_off (fact_bytes, fk_off and the
 * fact pointer multiples of 4); the dimension relation has n_dim rows of
 * dim_bytes bytes whose int64 key at byte pk_off equals the row number (the
 * dimension's index maps key k to row k).  `out` receives n_fact rows of
 * fact_bytes + dim_bytes bytes, each a fact row followed by the dimension row
 * its key names:
 *   DPG_JOIN_MOVE   DPG-move join (§4.2.1): out[i] = fact[i] || dim[fk_i],
 *                   the dimension rows moved into fact order by DPG.
 *   DPG_JOIN_SORT   DPG-sort join (§4.2.1): the (fk, i) pairs sorted by fk
 *                   (ties by fact row) and fact rows moved into that order by
 *                   DPG: out[j] = fact[i_j] || dim[fk_j].
 *   DPG_JOIN_DIRECT the MOVE result in one direct pass (baseline).
 * Untuned, MOVE and SORT retrieve on the L2-run plan (see dpg_retrieve),
 * except MOVE with dimension rows of 192 bytes and more, which takes the
 * 3-pass plan; DPG_VARIANT selects a plan, and a forced 2-pass plan falls
 * back to the 3-pass plan (join rows need INTERNAL).
 * A foreign key outside [0, n_dim), or a referenced dimension row whose key
 * differs from its row number, is reported by dpg_sync as DPG_ERANGE.  MOVE
 * and SORT catch an out-of-range key before writing `out`; MOVE also checks
 * dimension keys before writing; SORT and DIRECT check dimension keys as they
 * copy (then `out` is partly written).
 */
enum { DPG_JOIN_MOVE = 0, DPG_JOIN_SORT = 1, DPG_JOIN_DIRECT = 2 };
dpg_status dpg_fk_join(dpg_ctx* ctx, const void* fact, size_t n_fact, size_t fact_bytes, size_t fk_off,
                       const void* dim, size_t n_dim, size_t dim_bytes, size_t pk_off, void* out, int mode,
                       void* stream);

/*
 * Batched retrieval: `count` requests (a HOST array; its pointers are device
 * pointers), each dst_k[i] = src_k[rids_k[i]] as in dpg_retrieve, with uneven
 * record counts and record sizes: dpg_run_batch (below) with every request a
 * retrieval item.  Requests that read the same source table with the same
 * record size are retrieved together by one DPG pass, so each run of the
 * table is probed once per group (each rid is still checked against its own
 * request's n_src).  Stream-ordered: after one warm-up call at the same
 * sizes, a batch can be captured in a CUDA graph (the request tables are
 * staged in context-owned pinned memory that a replay reads again: do not
 * issue other batches on the context between capture and replay).  A bad rid
 * in any request leaves every destination untouched and is reported by
 * dpg_sync.
 */
typedef struct dpg_request {
  const void* src;      /* n_src records of rec_bytes bytes */
  size_t n_src;
  size_t rec_bytes;     /* 1 .. 65536 */
  size_t n;             /* rids in this request */
  const int32_t* rids;
  void* dst;            /* n records */
} dpg_request;

dpg_status dpg_retrieve_batch(dpg_ctx* ctx, const dpg_request* reqs, size_t count, void* stream);

/*
 * Serving (the paper has no serving layer; this runs its retrieval and joins
 * as a request loop).  A server owns `slots` execution slots (a context and a
 * stream each) on one device and a private stream-ordered memory pool.  Jobs
 * are queued in submission order; the head of the queue is admitted as soon
 * as a slot is free and the device memory held by running jobs and by results
 * not yet released, plus the job's own work space and result, fits within
 * budget_bytes.  While the head does not fit, the first later job that does
 * is admitted ahead of it, at most 4 x slots times per head (the environment
 * variable DPG_SERVE_BYPASS sets the bound; 0 keeps strict arrival order), so
 * a large job neither blocks small ones nor starves.  Admitted jobs run
 * concurrently; jobs that arrive while others
 * run are admitted as slots and memory free up (continuous batching).  A job's
 * tables are device pointers owned by the caller and must stay valid until
 * the job completes; its result is allocated by the server, read with
 * dpg_server_result and freed by dpg_server_release.
 */
typedef struct dpg_server dpg_server;
enum { DPG_JOB_RETRIEVE = 0, DPG_JOB_JOIN = 1 };
typedef struct dpg_job {
  int kind;             /* DPG_JOB_RETRIEVE or DPG_JOB_JOIN */
  int join_mode;        /* DPG_JOIN_* for joins */
  /* retrieval: result = n records, result[i] = src[rids[i]] (dpg_retrieve) */
  const void* src;
  size_t n_src;
  size_t rec_bytes;
  size_t n;
  const int32_t* rids;
  /* join: result = n_fact rows fact || dim (dpg_fk_join) */
  const void* fact;
  size_t n_fact;
  size_t fact_bytes;
  size_t fk_off;
  const void* dim;
  size_t n_dim;
  size_t dim_bytes;
  size_t pk_off;
} dpg_job;

/*
 * Batch execution (§2.1 and §4.2.1 for many requests at once; the paper has
 * no batch layer).  `count` items (a HOST array; its pointers are device
 * pointers), each a retrieval (job.kind DPG_JOB_RETRIEVE: out[i] =
 * src[rids[i]], n records of rec_bytes) or a DPG-move join (job.kind
 * DPG_JOB_JOIN, job.join_mode DPG_JOIN_MOVE: out row i = fact[i] ||
 * dim[fk_i], the layout rules of dpg_fk_join), of uneven sizes, run by a
 * persistent executor over a device table of work items (request group, DPG
 * phase, chunk) that its CTAs claim in order: persistent launches in stream
 * order, one per DPG phase for phases I (histogram and partition, two
 * kernels) and, for phases II and III, one per word size (4, 8 or 16 bytes)
 * of the groups that move records as 16-byte chunks plus one for the rest
 * (at most ten per call); or, with the environment variable
 * DPG_EXEC_FUSED=1, all phases in ONE persistent launch where an item
 * waits, with the context's wait limit (dpg_set_wait_limit), only for items
 * claimed before it.  Retrievals reading the same source table with the same record size
 * share one DPG pass over the L2-resident runs of that table (each rid is
 * still checked against its own n_src); a join is a group of its own.  Per
 * group the plan is the L2-run plan through INTERNAL below 192-byte records
 * and for joins, and the fused plan that writes each record straight to its
 * destination from 192 bytes, unless dpg_tune cached a plan for the group's
 * shape (its 2-pass plan maps to the fused plan, its L2-run and 3-pass plans
 * to the plan through INTERNAL).  Before anything is written every rid of every item is checked: a
 * bad rid or key anywhere leaves every destination untouched and dpg_sync
 * returns DPG_ERANGE (a dimension row whose key differs from its row number
 * is found later, as in dpg_fk_join).  Work space comes from the context (one
 * warm-up call at the same sizes before a CUDA-graph capture; the item
 * tables are staged in context-owned pinned memory that a replay reads
 * again).  Argument errors return DPG_EINVAL with nothing enqueued.
 */
typedef struct dpg_batch_item {
  dpg_job job;
  void* out;            /* n records, or n_fact join rows of fact_bytes + dim_bytes */
} dpg_batch_item;

dpg_status dpg_run_batch(dpg_ctx* ctx, const dpg_batch_item* items, size_t count, void* stream);

dpg_status dpg_server_create(dpg_server** out, int device, int slots, size_t budget_bytes);
/* Queue a job; *ticket identifies it.  DPG_EINVAL for a malformed job,
 * DPG_EBUSY when the job alone needs more than the budget. */
dpg_status dpg_server_submit(dpg_server* srv, const dpg_job* job, uint64_t* ticket);
/* The job's final status (as dpg_sync would report it), its result (device
 * pointer and size) and its latency from submission to completion.  With
 * wait == 0 returns DPG_EBUSY while the job is pending. */
dpg_status dpg_server_result(dpg_server* srv, uint64_t ticket, int wait, void** result, size_t* result_bytes,
                             double* latency_ms);
/* Free a completed job's result and forget the ticket.  The memory returns
 * to the server's pool in the order of the job's stream and may be handed to
 * the next job at once: work the caller enqueued on its own streams that
 * reads the result must have finished before this call. */
dpg_status dpg_server_release(dpg_server* srv, uint64_t ticket);
/* Device bytes currently held by running jobs and unreleased results. */
size_t dpg_server_held_bytes(dpg_server* srv);
/* Finish running jobs (queued ones are dropped), free everything. */
void dpg_server_destroy(dpg_server* srv);

/* Blocks until `stream` has finished, then returns the first asynchronous
 * error raised by this context's kernels since the previous dpg_sync
 * (DPG_ERANGE, DPG_ETIMEOUT) and clears it; DPG_OK when there was none. */
dpg_status dpg_sync(dpg_ctx* ctx, void* stream);

/* Number of kernels this context has launched since it was created. */
uint64_t dpg_kernel_launches(dpg_ctx* ctx);

/*
 * Failure detection (the paper has none; these bound and exercise the
 * library's own device-side waits).
 *
 * dpg_set_wait_limit: every wait of this context's kernels on a flag that
 * another CTA writes (the radix sort's look-back over earlier tiles, the
 * batch executor's waits for a request's earlier phase) gives up after
 * `seconds` of SM clock (default about 1 s), sets the timeout bit and lets
 * the kernel return; the next dpg_sync reports DPG_ETIMEOUT.  Results of a
 * call whose wait ran out are undefined, but every write stays inside the
 * call's own buffers and the context stays usable.  0 < seconds <= 60, else
 * DPG_EINVAL.
 *
 * dpg_check_wait: enqueues one kernel that waits, under the context's limit,
 * on a device word that nothing ever sets; the following dpg_sync returns
 * DPG_ETIMEOUT once the limit has passed.  It runs the same bounded wait the
 * sort and the batch executor use, so a caller (or a test) can see a wait
 * run out without faulting or hanging the GPU.
 *
 * dpg_inject_alloc_failure: the next `count` device allocations of this
 * context (scratch, work space, host-call buffers) fail as if cudaMalloc had
 * failed: the call that needed one returns DPG_ENOMEM having enqueued
 * nothing and left its destination untouched.  count 0 clears it.
 */
dpg_status dpg_set_wait_limit(dpg_ctx* ctx, double seconds);
dpg_status dpg_check_wait(dpg_ctx* ctx, void* stream);
dpg_status dpg_inject_alloc_failure(dpg_ctx* ctx, int count);

/*
 * Host-buffer variants (the paper states retrieval between files, §1; here
 * the "files" are host memory).  src/pairs, rids and dst are HOST pointers
 * (page-locked memory gives full copy bandwidth).  The call copies the inputs
 * into context-owned device buffers, runs the device entry point of the same
 * name, copies the result back and synchronizes `stream`; it returns the final
 * status, DPG_ERANGE included (dst untouched then).
 */
dpg_status dpg_retrieve_host(dpg_ctx* ctx, const void* src, size_t n_src, size_t rec_bytes, size_t n,
                             const int32_t* rids, void* dst, void* stream);
dpg_status dpg_sort_copy_host(dpg_ctx* ctx, const void* pairs, size_t pair_stride, size_t rid_off,
                              size_t n, const void* src, size_t n_src, size_t rec_bytes, void* dst,
                              void* stream);

/*
 * Plan tuning (the paper fixes the run length to half the cache, §2.1; on a
 * GPU the best run length and plan depend on the record size and the table
 * sizes, so they are measured).  dpg_tune runs each candidate plan for this
 * retrieval shape on the caller's data (rids at rid_base, rid_stride bytes
 * apart: 4 for an int32 array, 16 with rid_off 12 for key-pointer pairs;
 * dst receives the result), times them with CUDA events on `stream`, and
 * caches the fastest in the context for retrievals of the same record size,
 * size classes (log2 of n_src and n) and rid layout.  Blocking.  Candidates:
 * the 3-pass plan with shared-memory segments of the largest power-of-two
 * record count that fits 104 KB and of one half and one quarter of it, the
 * 2-pass plan, and the L2-run plan with runs of about 4, 8 and 16 MB.
 * *variant (3, 2 or 4) and *seg_log2 receive the winner (may be NULL).
 * dpg_last_plan reports the plan of the context's last retrieval.
 */
dpg_status dpg_tune(dpg_ctx* ctx, const void* src, size_t n_src, size_t rec_bytes, size_t n, const void* rid_base,
                    size_t rid_stride, void* dst, void* stream, int* variant, int* seg_log2);
void dpg_last_plan(dpg_ctx* ctx, int* variant, int* seg_log2);

/*
 * Kernel tracing (measurement support; the paper has none).  While enabled,
 * every kernel the context launches is bracketed by two CUDA events recorded
 * on its stream.  dpg_trace_count / dpg_trace_get wait for the recorded
 * events and report, per kernel name, the summed event time in milliseconds
 * and the number of launches since the last dpg_trace_reset.  Names are owned
 * by the context and stay valid until dpg_trace_reset or dpg_ctx_destroy.
 */
void dpg_trace_enable(dpg_ctx* ctx, int on);
void dpg_trace_reset(dpg_ctx* ctx);
size_t dpg_trace_count(dpg_ctx* ctx);
dpg_status dpg_trace_get(dpg_ctx* ctx, size_t index, const char** name, double* total_ms,
                         uint64_t* launches);

/*
 * Allocation-free retrieval.  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory at the time of the call (code
 * running while a caching allocator holds all free memory, memory-capped or
 * pre-budgeted regions, plug-ins that must not allocate after start-up).
 *
 * Same result as dpg_retrieve (dst[i] = src[rids[i]], computed by the 2-pass
 * DPG plan), but it takes no context and allocates nothing: its scratch is a
 * fixed ~17.7 MB array that the library reserves on every device it is loaded
 * on, until the process exits.  Runs on the calling thread's current device;
 * all pointers are device pointers on that device.
 *   - Limits: n <= 2,097,152 rids, rec_bytes <= 65536, and at most 4096
 *     source segments of up to 104 KB each (about 420 MB of 100-byte records);
 *     beyond them it returns DPG_EINVAL and enqueues nothing.
 *   - The first call on each device does the set-up: it looks up the
 *     array's device address, and if no other call of this library has run
 *     on that device yet, the CUDA runtime loads the library's device code
 *     there (modules load lazily), which is when the array is reserved.  So
 *     make the first call at start-up, before a caching allocator or a
 *     memory cap takes the free memory, and before any stream capture.
 *     Later calls allocate nothing.
 *   - The call is synchronous: it waits for `stream` and returns the final
 *     status (DPG_ERANGE for a bad rid, destination untouched).
 *   - Every call uses the same array (each call clears what must start at
 *     zero): calls whose GPU work overlaps, from two streams or two host
 *     threads, race and may return wrong data.
 */
dpg_status dpg_retrieve_noalloc(const void* src, size_t n_src, size_t rec_bytes, size_t n,
                                const int32_t* rids, void* dst, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DPG_H */
