/*
 * Seeded synthetic input generators shared by the tests, the oracle's
 * callers and bench.py.  This file holds no arithmetic of the retrieval
 * method: it only produces source records, rid sequences and foreign keys.
 *
 * Every stream is SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): state s_0 = seed,
 * s_k = s_{k-1} + 0x9e3779b97f4a7c15, output_k = mix(s_k), k = 1, 2, ...
 * Because output_k depends only on (seed, k), the byte fill and the
 * independent draws are generated in parallel chunks that reproduce the
 * sequential stream exactly.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* k-th output (k >= 1) of SplitMix64 started at `seed`. */
uint64_t synth_splitmix64_at(uint64_t seed, uint64_t k) { return mix64(seed + k * GOLDEN); }

/* Seed of an independent sub-stream: the (stream+1)-th output of seed's stream. */
uint64_t synth_stream_seed(uint64_t seed, uint64_t stream) { return mix64(seed + (stream + 1) * GOLDEN); }

/* floor(x * m / 2^64): an unbiased-enough map of a 64-bit draw into [0, m). */
static inline uint64_t mulhi_range(uint64_t x, uint64_t m) {
  return (uint64_t)(((unsigned __int128)x * m) >> 64);
}

/* Fill buf[0, nbytes) with successive outputs of SplitMix64(seed) stored
 * little-endian; the final partial word is truncated. */
void synth_fill_bytes(uint8_t* buf, uint64_t nbytes, uint64_t seed) {
  uint64_t nwords = nbytes / 8;
#pragma omp parallel for schedule(static)
  for (int64_t w = 0; w < (int64_t)nwords; ++w) {
    uint64_t v = mix64(seed + (uint64_t)(w + 1) * GOLDEN);
    for (int b = 0; b < 8; ++b) buf[(uint64_t)w * 8 + b] = (uint8_t)(v >> (8 * b));
  }
  uint64_t rem = nbytes - nwords * 8;
  if (rem) {
    uint64_t v = mix64(seed + (nwords + 1) * GOLDEN);
    for (uint64_t b = 0; b < rem; ++b) buf[nwords * 8 + b] = (uint8_t)(v >> (8 * b));
  }
}

/* Fisher-Yates shuffle of the identity on [0, n): for i = n-1 down to 1,
 * j = floor(draw * (i+1) / 2^64), swap p[i], p[j]; draws are consecutive
 * outputs of SplitMix64(seed). */
void synth_permutation_i32(int32_t* p, uint64_t n, uint64_t seed) {
  for (uint64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
  uint64_t s = seed;
  for (uint64_t i = n; i-- > 1;) {
    s += GOLDEN;
    uint64_t j = mulhi_range(mix64(s), i + 1);
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
}

/* Uniform draws with replacement: out[k] = floor(output_{k+1} * m / 2^64). */
void synth_uniform_i32(int32_t* out, uint64_t n, uint64_t m, uint64_t seed) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)n; ++k)
    out[k] = (int32_t)mulhi_range(mix64(seed + (uint64_t)(k + 1) * GOLDEN), m);
}

/* Uniform doubles in [0,1): top 53 bits of each draw. */
void synth_uniform_f64(double* out, uint64_t n, uint64_t seed) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)n; ++k)
    out[k] = (double)(mix64(seed + (uint64_t)(k + 1) * GOLDEN) >> 11) * 0x1.0p-53;
}

/* Zipf(s) over ranks 1..K by inverse CDF: cdf[k-1] = sum_{j<=k} j^-s / H,
 * rank = smallest k with u < cdf[k-1]; u = top 53 bits of each draw.
 * Writes rank-1 (0-based) into out. */
int synth_zipf_i32(int32_t* out, uint64_t n, uint64_t K, double s, uint64_t seed) {
  if (K == 0) return 1;
  double* cdf = (double*)malloc(K * sizeof(double));
  if (!cdf) return 2;
  double acc = 0.0;
  for (uint64_t k = 1; k <= K; ++k) { acc += pow((double)k, -s); cdf[k - 1] = acc; }
  for (uint64_t k = 0; k < K; ++k) cdf[k] /= acc;
  cdf[K - 1] = 1.0;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < (int64_t)n; ++t) {
    double u = (double)(mix64(seed + (uint64_t)(t + 1) * GOLDEN) >> 11) * 0x1.0p-53;
    uint64_t lo = 0, hi = K - 1;           /* first index with u < cdf[idx] */
    while (lo < hi) { uint64_t mid = lo + (hi - lo) / 2; if (u < cdf[mid]) hi = mid; else lo = mid + 1; }
    out[t] = (int32_t)lo;
  }
  free(cdf);
  return 0;
}

/* out[k] = table[idx[k]] (used to push Zipf ranks through a shuffle). */
void synth_take_i32(int32_t* out, const int32_t* idx, const int32_t* table, uint64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)n; ++k) out[k] = table[idx[k]];
}

/* Rid lists of a batch of requests, each from its own sub-stream of `seed`:
 * request k writes n[k] rids at out + offset[k]; kind[k] = 1: a Fisher-Yates
 * permutation of [0, n[k]) (requires n_src[k] == n[k]), kind[k] = 0: uniform
 * draws with replacement from [0, n_src[k]).  Requests run in parallel. */
void synth_batch_rids(int32_t* out, const uint64_t* offset, const uint64_t* n, const uint64_t* n_src,
                      const uint8_t* kind, uint64_t count, uint64_t seed) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < (int64_t)count; ++k) {
    const uint64_t s = synth_stream_seed(seed, (uint64_t)k);
    if (kind[k]) synth_permutation_i32(out + offset[k], n[k], s);
    else {
      for (uint64_t t = 0; t < n[k]; ++t) out[offset[k] + t] = (int32_t)mulhi_range(mix64(s + (t + 1) * GOLDEN), n_src[k]);
    }
  }
}
