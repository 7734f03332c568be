/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, obviously correct CPU statement of what the record-retrieval
 * path computes, written from Cooperman, Ma and Nguyen, "DPG: A Cache-Efficient
 * Accelerator for Sorting and for Join Operators" (cs/0308004).  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * CUDA library never does, and this file shares no code with it.
 *
 * All work here is integer and byte movement: results are unique and compared
 * byte for byte.  Status codes: 0 = ok, 1 = invalid argument, 2 = a rid or
 * foreign key outside its table (nothing written).
 *
 * Pins (tests/test_oracle_pins.py): brute force over all permutations of small
 * rid sequences against an inverse-permutation formulation; decoding of
 * self-describing records (each record carries its own index) for duplicates,
 * exactly-once and multiset invariants; the worked example of §2.2; agreement
 * of the three-phase statement (§2.1) with the one-line definition (§2);
 * sortedness + permutation + tie order for the key-pointer sort (§3);
 * nested-loop agreement for the foreign-key joins (§4.2).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_EINVAL = 1, OR_ERANGE = 2, OR_ENOMEM = 3 };

/* §2 (the "for each i, D[i] = R[S_rid[i]]" statement) and §1 (the record
 * retrieval problem): copy source record rids[i] to destination slot i.
 * Every rid must lie in [0, n_src) (§2.1 assumes rid values between 0 and N);
 * they are all checked before the first byte is written. */
int oracle_retrieve(const uint8_t* src, uint64_t n_src, uint64_t rec, uint64_t n,
                    const int32_t* rids, uint8_t* dst) {
  if (rec == 0) return OR_EINVAL;
  for (uint64_t i = 0; i < n; ++i)
    if (rids[i] < 0 || (uint64_t)rids[i] >= n_src) return OR_ERANGE;
  for (uint64_t i = 0; i < n; ++i)
    memcpy(dst + i * rec, src + (uint64_t)rids[i] * rec, rec);
  return OR_OK;
}

/* The same retrieval on `threads` POSIX threads, for the benchmark's
 * multi-core CPU figure: the threads first check the rids of their own
 * contiguous ranges of destination slots and, only if every rid of every range
 * is in [0, n_src), then copy those ranges.  The tests check it against
 * oracle_retrieve. */
struct or_range {
  const uint8_t* src;
  uint64_t n_src, rec, lo, hi;
  const int32_t* rids;
  uint8_t* dst;
  int bad;
};

static void* or_check_range(void* arg) {
  struct or_range* r = (struct or_range*)arg;
  for (uint64_t i = r->lo; i < r->hi; ++i)
    if (r->rids[i] < 0 || (uint64_t)r->rids[i] >= r->n_src) r->bad = 1;
  return NULL;
}

static void* or_copy_range(void* arg) {
  struct or_range* r = (struct or_range*)arg;
  for (uint64_t i = r->lo; i < r->hi; ++i)
    memcpy(r->dst + i * r->rec, r->src + (uint64_t)r->rids[i] * r->rec, r->rec);
  return NULL;
}

static int or_run_ranges(struct or_range* ranges, pthread_t* tids, uint64_t threads, void* (*fn)(void*)) {
  uint64_t started = 0;
  int rc = OR_OK;
  for (; started < threads; ++started)
    if (pthread_create(&tids[started], NULL, fn, &ranges[started]) != 0) {
      rc = OR_ENOMEM;
      break;
    }
  for (uint64_t t = 0; t < started; ++t) pthread_join(tids[t], NULL);
  return rc;
}

int oracle_retrieve_threads(const uint8_t* src, uint64_t n_src, uint64_t rec, uint64_t n,
                            const int32_t* rids, uint8_t* dst, uint64_t threads) {
  if (rec == 0 || threads == 0) return OR_EINVAL;
  if (threads > n) threads = n ? n : 1;
  struct or_range* ranges = calloc(threads, sizeof *ranges);
  pthread_t* tids = calloc(threads, sizeof *tids);
  if (!ranges || !tids) {
    free(ranges);
    free(tids);
    return OR_ENOMEM;
  }
  for (uint64_t t = 0; t < threads; ++t) {
    ranges[t] = (struct or_range){src, n_src, rec, n * t / threads, n * (t + 1) / threads, rids, dst, 0};
  }
  int rc = or_run_ranges(ranges, tids, threads, or_check_range);
  for (uint64_t t = 0; rc == OR_OK && t < threads; ++t)
    if (ranges[t].bad) rc = OR_ERANGE;
  if (rc == OR_OK) rc = or_run_ranges(ranges, tids, threads, or_copy_range);
  free(ranges);
  free(tids);
  return rc;
}

/* §2.1, stated as the three results its phases produce (small inputs only:
 * the cost is quadratic).  Runs are numbered from 0 and run j covers source
 * records [j*L, (j+1)*L).
 *   Phase I result, the RID runs: run j is the subsequence of the rid list
 *            formed by the rids r with r div L = j, in list order.
 *   Phase II result, INTERNAL: entry k of the runs laid end to end (run 0
 *            first) is the source record that rid entry k names.
 *   Phase III result, OUTPUT: the record of rid i is the INTERNAL entry at
 *            the start of its run j = rids[i] div L plus the number of rids
 *            before i in the list that also fall in run j.
 * Outputs: rid_runs (n rids, runs end to end), run_sizes (ceil(n_src / L)
 * counts), internal (n records), dst (n records).  A run holds as many
 * entries as rids fall in it, duplicates and skew included (§2, §2.3). */
int oracle_dpg_phases(const uint8_t* src, uint64_t n_src, uint64_t rec, uint64_t n,
                      const int32_t* rids, uint64_t L, int32_t* rid_runs, uint64_t* run_sizes,
                      uint8_t* internal, uint8_t* dst) {
  if (rec == 0 || L == 0) return OR_EINVAL;
  for (uint64_t i = 0; i < n; ++i)
    if (rids[i] < 0 || (uint64_t)rids[i] >= n_src) return OR_ERANGE;
  uint64_t num_runs = (n_src + L - 1) / L;
  /* RID runs: for each run, select its rids from the whole list, in order. */
  uint64_t pos = 0;
  for (uint64_t j = 0; j < num_runs; ++j) {
    run_sizes[j] = 0;
    for (uint64_t i = 0; i < n; ++i)
      if ((uint64_t)rids[i] / L == j) {
        rid_runs[pos++] = rids[i];
        run_sizes[j]++;
      }
  }
  /* INTERNAL: the record each run entry names. */
  for (uint64_t k = 0; k < n; ++k)
    memcpy(internal + k * rec, src + (uint64_t)rid_runs[k] * rec, rec);
  /* OUTPUT: rid i's entry = start of its run + its rank among that run's rids. */
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t j = (uint64_t)rids[i] / L, start = 0, rank = 0;
    for (uint64_t m = 0; m < j; ++m) start += run_sizes[m];
    for (uint64_t m = 0; m < i; ++m)
      if ((uint64_t)rids[m] / L == j) rank++;
    memcpy(dst + i * rec, internal + (start + rank) * rec, rec);
  }
  return OR_OK;
}

/* ---- §3: three-phase sort (extract key-pointer pairs, sort them, copy). ---- */

/* Key-pointer pair layout: bytes [0, key_bytes) the record's key, zero padding
 * up to byte 12, then the int32 rid little-endian at byte 12.  16 bytes. */
#define OR_PAIR 16
#define OR_RID_OFF 12

static uint64_t g_key_bytes;  /* comparator parameter (the oracle is single-threaded) */

static int32_t pair_rid(const uint8_t* p) {
  int32_t r; memcpy(&r, p + OR_RID_OFF, 4); return r;
}

/* Order: keys as unsigned byte strings (memcmp), equal keys by ascending rid. */
static int cmp_pair(const void* a, const void* b) {
  int c = memcmp(a, b, g_key_bytes);
  if (c) return c;
  int32_t ra = pair_rid((const uint8_t*)a), rb = pair_rid((const uint8_t*)b);
  return (ra > rb) - (ra < rb);
}

/* Phases 1 and 2 of §3: pairs[i] = (key of record i, i), then sorted. */
int oracle_sort_keyptr(const uint8_t* src, uint64_t n_src, uint64_t rec, uint64_t key_bytes,
                       uint8_t* pairs) {
  if (rec == 0 || key_bytes == 0 || key_bytes > OR_RID_OFF || key_bytes > rec) return OR_EINVAL;
  if (n_src > 0x80000000ULL) return OR_EINVAL;
  memset(pairs, 0, n_src * OR_PAIR);
  for (uint64_t i = 0; i < n_src; ++i) {
    memcpy(pairs + i * OR_PAIR, src + i * rec, key_bytes);
    int32_t r = (int32_t)i;
    memcpy(pairs + i * OR_PAIR + OR_RID_OFF, &r, 4);
  }
  g_key_bytes = key_bytes;
  qsort(pairs, n_src, OR_PAIR, cmp_pair);
  return OR_OK;
}

/* Phase 3 of §3: record retrieval with the rids read out of the sorted pairs
 * (each pair is `stride` bytes, its rid an int32 at byte rid_off). */
int oracle_sort_copy(const uint8_t* pairs, uint64_t stride, uint64_t rid_off, uint64_t n,
                     const uint8_t* src, uint64_t n_src, uint64_t rec, uint8_t* dst) {
  if (rec == 0 || stride < 4 || rid_off + 4 > stride) return OR_EINVAL;
  for (uint64_t i = 0; i < n; ++i) {
    int32_t r; memcpy(&r, pairs + i * stride + rid_off, 4);
    if (r < 0 || (uint64_t)r >= n_src) return OR_ERANGE;
  }
  for (uint64_t i = 0; i < n; ++i) {
    int32_t r; memcpy(&r, pairs + i * stride + rid_off, 4);
    memcpy(dst + i * rec, src + (uint64_t)r * rec, rec);
  }
  return OR_OK;
}

/* ---- §4.2: foreign-key join of a fact relation (rows carry an int32 foreign
 * key at fk_off) with a dimension relation (rows carry an int64 key at pk_off).
 * Output rows are fact row || dimension row. ---- */

static int64_t rd_i64(const uint8_t* p) { int64_t v; memcpy(&v, p, 8); return v; }
static int32_t rd_i32(const uint8_t* p) { int32_t v; memcpy(&v, p, 4); return v; }

/* The textbook join: for each fact row in file order, for each dimension row
 * in file order, emit the concatenation when the keys are equal.  Quadratic;
 * small inputs only.  *out_rows receives the number of rows emitted; rows past
 * out_cap are counted but not written. */
int oracle_fk_join_nested(const uint8_t* fact, uint64_t n_fact, uint64_t fact_bytes, uint64_t fk_off,
                          const uint8_t* dim, uint64_t n_dim, uint64_t dim_bytes, uint64_t pk_off,
                          uint8_t* out, uint64_t out_cap, uint64_t* out_rows) {
  if (fk_off + 4 > fact_bytes || pk_off + 8 > dim_bytes) return OR_EINVAL;
  uint64_t w = fact_bytes + dim_bytes, k = 0;
  for (uint64_t i = 0; i < n_fact; ++i) {
    int64_t fk = rd_i32(fact + i * fact_bytes + fk_off);
    for (uint64_t d = 0; d < n_dim; ++d) {
      if (rd_i64(dim + d * dim_bytes + pk_off) == fk) {
        if (k < out_cap) {
          memcpy(out + k * w, fact + i * fact_bytes, fact_bytes);
          memcpy(out + k * w + fact_bytes, dim + d * dim_bytes, dim_bytes);
        }
        ++k;
      }
    }
  }
  *out_rows = k;
  return OR_OK;
}

/* DPG-move join output (§4.2.1, goal 1): dimension rows moved into fact order.
 * The dimension's index maps key k to row k (its primary key is the row
 * number), so rid_F = fk; the pair is checked against the stored key. */
int oracle_fk_join_move(const uint8_t* fact, uint64_t n_fact, uint64_t fact_bytes, uint64_t fk_off,
                        const uint8_t* dim, uint64_t n_dim, uint64_t dim_bytes, uint64_t pk_off,
                        uint8_t* out) {
  if (fk_off + 4 > fact_bytes || pk_off + 8 > dim_bytes) return OR_EINVAL;
  for (uint64_t i = 0; i < n_fact; ++i) {
    int32_t fk = rd_i32(fact + i * fact_bytes + fk_off);
    if (fk < 0 || (uint64_t)fk >= n_dim) return OR_ERANGE;
    if (rd_i64(dim + (uint64_t)fk * dim_bytes + pk_off) != fk) return OR_ERANGE;
  }
  uint64_t w = fact_bytes + dim_bytes;
  for (uint64_t i = 0; i < n_fact; ++i) {
    int32_t fk = rd_i32(fact + i * fact_bytes + fk_off);
    memcpy(out + i * w, fact + i * fact_bytes, fact_bytes);
    memcpy(out + i * w + fact_bytes, dim + (uint64_t)fk * dim_bytes, dim_bytes);
  }
  return OR_OK;
}

typedef struct { int32_t fk; int32_t pad; uint64_t i; } or_rid_pair;

static int cmp_rid_pair(const void* a, const void* b) {
  const or_rid_pair *x = (const or_rid_pair*)a, *y = (const or_rid_pair*)b;
  if (x->fk != y->fk) return (x->fk > y->fk) - (x->fk < y->fk);
  return (x->i > y->i) - (x->i < y->i);
}

/* DPG-sort join output (§4.2.1, goal 2): the rid pairs (rid_R = fact row,
 * rid_F = fk) sorted by rid_F, equal rid_F by rid_R, and fact rows moved into
 * that order; each output row is fact row || its dimension row. */
int oracle_fk_join_sorted(const uint8_t* fact, uint64_t n_fact, uint64_t fact_bytes, uint64_t fk_off,
                          const uint8_t* dim, uint64_t n_dim, uint64_t dim_bytes, uint64_t pk_off,
                          uint8_t* out) {
  if (fk_off + 4 > fact_bytes || pk_off + 8 > dim_bytes) return OR_EINVAL;
  for (uint64_t i = 0; i < n_fact; ++i) {
    int32_t fk = rd_i32(fact + i * fact_bytes + fk_off);
    if (fk < 0 || (uint64_t)fk >= n_dim) return OR_ERANGE;
    if (rd_i64(dim + (uint64_t)fk * dim_bytes + pk_off) != fk) return OR_ERANGE;
  }
  or_rid_pair* p = (or_rid_pair*)malloc((n_fact ? n_fact : 1) * sizeof(or_rid_pair));
  if (!p) return OR_ENOMEM;
  for (uint64_t i = 0; i < n_fact; ++i) { p[i].fk = rd_i32(fact + i * fact_bytes + fk_off); p[i].pad = 0; p[i].i = i; }
  qsort(p, n_fact, sizeof(or_rid_pair), cmp_rid_pair);
  uint64_t w = fact_bytes + dim_bytes;
  for (uint64_t k = 0; k < n_fact; ++k) {
    memcpy(out + k * w, fact + p[k].i * fact_bytes, fact_bytes);
    memcpy(out + k * w + fact_bytes, dim + (uint64_t)p[k].fk * dim_bytes, dim_bytes);
  }
  free(p);
  return OR_OK;
}

/* The fact-row order of the DPG-sort join (§4.2.1): the row indices of the
 * fact relation ordered by foreign key, equal keys by row index, found by a
 * stable counting sort over the key range [0, n_dim) (every key is checked
 * first).  order receives n_fact indices.  Linear time, so it serves the
 * full-size join: out row j of the sorted join is the DPG-move row of fact
 * row order[j].  The tests pin it to oracle_fk_join_sorted. */
int oracle_fk_join_order(const uint8_t* fact, uint64_t n_fact, uint64_t fact_bytes, uint64_t fk_off,
                         uint64_t n_dim, uint64_t* order) {
  if (fk_off + 4 > fact_bytes) return OR_EINVAL;
  for (uint64_t i = 0; i < n_fact; ++i) {
    int32_t fk = rd_i32(fact + i * fact_bytes + fk_off);
    if (fk < 0 || (uint64_t)fk >= n_dim) return OR_ERANGE;
  }
  uint64_t* start = (uint64_t*)calloc(n_dim + 1, sizeof(uint64_t));
  if (!start) return OR_ENOMEM;
  for (uint64_t i = 0; i < n_fact; ++i) start[(uint64_t)rd_i32(fact + i * fact_bytes + fk_off) + 1]++;
  for (uint64_t k = 0; k < n_dim; ++k) start[k + 1] += start[k];  /* start[k] = rows with a smaller key */
  for (uint64_t i = 0; i < n_fact; ++i) order[start[(uint64_t)rd_i32(fact + i * fact_bytes + fk_off)]++] = i;
  free(start);
  return OR_OK;
}
