/*
 * Seeded synthetic sparse document collections (inputs only).
 *
 * This file produces the object set X-hat of the paper's problem statement
 * (Section 2.3, Fig. 1: each object is an array of (term id, value) tuples),
 * shaped like its tf-idf corpora (Section 5.1): Zipf-distributed term ids
 * without repeats inside a document, lognormal weights, each document
 * L2-normalised.  It holds none of the clustering method's arithmetic and is
 * shared by the FP64 oracle and the CUDA path alike.
 *
 * Randomness is counter based: every document owns a stream
 *   u_n = mix(base(seed, doc, purpose) + n * 0x9E3779B97F4A7C15)
 * where mix is the SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014).
 * A document's bytes therefore depend only on (seed, doc index), never on the
 * thread count or scheduling.  Compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PURPOSE_LENGTH 1u
#define PURPOSE_TERMS 2u

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t base;
  uint64_t n;
} stream_t;

static inline stream_t open_stream(uint64_t seed, uint64_t doc, uint64_t purpose) {
  stream_t s;
  s.base = mix64(mix64(seed + 0x632BE59BD9B4E019ULL) ^ (doc * 0xD1B54A32D192ED03ULL + purpose));
  s.n = 0;
  return s;
}

static inline uint64_t next_u64(stream_t* s) {
  s->n += 1;
  return mix64(s->base + s->n * 0x9E3779B97F4A7C15ULL);
}

/* uniform in [0, 1) with 53 random bits */
static inline double next_unit(stream_t* s) { return (double)(next_u64(s) >> 11) * 0x1.0p-53; }

/* standard normal by the Box-Muller transform */
static inline double next_normal(stream_t* s) {
  double u1 = 1.0 - next_unit(s); /* (0, 1] */
  double u2 = next_unit(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Poisson(lambda) by inversion of the CDF, walking up from k = 0 */
static int64_t next_poisson(stream_t* s, double lambda) {
  double u = next_unit(s);
  double p = exp(-lambda), f = p;
  int64_t k = 0;
  while (u > f && k < 100000) {
    k += 1;
    p *= lambda / (double)k;
    f += p;
    if (p == 0.0 && f < u) break; /* numerically exhausted tail */
  }
  return k;
}

/*
 * Document lengths (number of distinct terms).
 *   kind 0: Poisson(param) clipped to [lo, hi]
 *   kind 1: round(lognormal(ln(param) - sigma^2/2, sigma)) clipped to [lo, hi]
 *           (so the unclipped mean is `param`)
 * hi is also capped at n_terms.  Returns 0, or -1 on bad arguments.
 */
int corpus_lengths(int64_t n_docs, int64_t n_terms, int kind, double param, double sigma,
                   int64_t lo, int64_t hi, uint64_t seed, int64_t* lengths) {
  if (n_docs < 0 || n_terms < 1 || lo < 1 || hi < lo || !lengths) return -1;
  if (hi > n_terms) hi = n_terms;
  if (lo > hi) lo = hi;
  double mu = (kind == 1) ? log(param) - 0.5 * sigma * sigma : 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t d = 0; d < n_docs; ++d) {
    stream_t s = open_stream(seed, (uint64_t)d, PURPOSE_LENGTH);
    int64_t L;
    if (kind == 0) {
      L = next_poisson(&s, param);
    } else {
      double z = next_normal(&s);
      L = (int64_t)llround(exp(mu + sigma * z));
    }
    if (L < lo) L = lo;
    if (L > hi) L = hi;
    lengths[d] = L;
  }
  return 0;
}

/* truncated Zipf CDF over ranks 1..n_terms with exponent s; cdf[n_terms-1] == 1 */
int corpus_zipf_cdf(int64_t n_terms, double s, double* cdf) {
  if (n_terms < 1 || !cdf) return -1;
  double acc = 0.0;
  for (int64_t r = 0; r < n_terms; ++r) {
    acc += pow((double)(r + 1), -s);
    cdf[r] = acc;
  }
  for (int64_t r = 0; r < n_terms; ++r) cdf[r] /= acc;
  cdf[n_terms - 1] = 1.0;
  return 0;
}

/* smallest r with cdf[r] > u (u in [0,1)) */
static inline int64_t zipf_rank(const double* cdf, int64_t n, double u) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (cdf[mid] > u)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

typedef struct {
  int32_t t;
  double v;
} entry_t;

static int cmp_entry(const void* a, const void* b) {
  int32_t x = ((const entry_t*)a)->t, y = ((const entry_t*)b)->t;
  return (x > y) - (x < y);
}

/*
 * Fill the CSR rows: row d gets row_ptr[d+1]-row_ptr[d] distinct term ids
 * drawn from the truncated Zipf law (rank r -> term id r-1, so frequent terms
 * get small ids; repeats inside a row are rejected and redrawn), each with a
 * lognormal(0, 1) weight; the row is sorted by term id and divided by its L2
 * norm (accumulated in FP64 in ascending term order), then stored as FP32.
 * If a row cannot collect its distinct terms within 1000 draws per term, the
 * smallest unused term ids complete it.  Returns 0, or -1 on bad arguments.
 */
int corpus_fill(int64_t n_docs, int64_t n_terms, const double* cdf, uint64_t seed,
                const int64_t* row_ptr, int32_t* term, float* val) {
  if (n_docs < 0 || n_terms < 1 || !cdf || !row_ptr || !term || !val) return -1;
  int64_t lmax = 0;
  for (int64_t d = 0; d < n_docs; ++d) {
    int64_t L = row_ptr[d + 1] - row_ptr[d];
    if (L < 0 || L > n_terms) return -1;
    if (L > lmax) lmax = L;
  }
  int64_t hcap = 16;
  while (hcap < 4 * lmax) hcap <<= 1;
  int bad = 0;
#pragma omp parallel
  {
    int32_t* table = (int32_t*)malloc((size_t)hcap * sizeof(int32_t));
    entry_t* ent = (entry_t*)malloc((size_t)(lmax > 0 ? lmax : 1) * sizeof(entry_t));
    if (!table || !ent) {
#pragma omp atomic write
      bad = 1;
    } else {
      for (int64_t i = 0; i < hcap; ++i) table[i] = -1;
#pragma omp for schedule(dynamic, 64)
      for (int64_t d = 0; d < n_docs; ++d) {
        int64_t L = row_ptr[d + 1] - row_ptr[d];
        stream_t s = open_stream(seed, (uint64_t)d, PURPOSE_TERMS);
        int64_t got = 0, draws = 0, budget = 1000 * (L + 1);
        while (got < L && draws < budget) {
          int32_t t = (int32_t)zipf_rank(cdf, n_terms, next_unit(&s));
          ++draws;
          uint64_t h = mix64((uint64_t)t) & (uint64_t)(hcap - 1);
          int dup = 0;
          while (table[h] >= 0) {
            if (table[h] == t) {
              dup = 1;
              break;
            }
            h = (h + 1) & (uint64_t)(hcap - 1);
          }
          if (dup) continue;
          table[h] = t;
          ent[got].t = t;
          ent[got].v = exp(next_normal(&s)); /* lognormal(0, 1) */
          ++got;
        }
        for (int32_t t = 0; got < L; ++t) { /* deterministic completion */
          uint64_t h = mix64((uint64_t)t) & (uint64_t)(hcap - 1);
          int dup = 0;
          while (table[h] >= 0) {
            if (table[h] == t) {
              dup = 1;
              break;
            }
            h = (h + 1) & (uint64_t)(hcap - 1);
          }
          if (dup) continue;
          table[h] = t;
          ent[got].t = t;
          ent[got].v = exp(next_normal(&s));
          ++got;
        }
        /* clear only the slots this row used (the scan skips emptied slots) */
        for (int64_t q = 0; q < L; ++q) {
          uint64_t h = mix64((uint64_t)ent[q].t) & (uint64_t)(hcap - 1);
          while (table[h] != ent[q].t) h = (h + 1) & (uint64_t)(hcap - 1);
          table[h] = -1;
        }
        qsort(ent, (size_t)L, sizeof(entry_t), cmp_entry);
        double ss = 0.0;
        for (int64_t q = 0; q < L; ++q) ss += ent[q].v * ent[q].v;
        double nrm = sqrt(ss);
        int64_t o = row_ptr[d];
        for (int64_t q = 0; q < L; ++q) {
          term[o + q] = ent[q].t;
          val[o + q] = (float)(ent[q].v / nrm);
        }
      }
    }
    free(table);
    free(ent);
  }
  return bad ? -1 : 0;
}
