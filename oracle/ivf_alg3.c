/*
 * Algorithm 3 (IVF) of arXiv 2002.09094 in plain C, FP64 -- test
 * infrastructure and the timed "paper's method on CPU" baseline.
 *
 * Only the tests, the smoke check and the benchmark's CPU legs load this
 * library; the CUDA path shares nothing with it.  It computes exactly what
 * oracle/inverted_file.py computes, in the same order of FP64 operations
 * (compile with -ffp-contract=off so no multiply-add is fused), so the two
 * agree bit for bit; the tests pin that and pin the Python module to the
 * paper's definitions.
 *
 * Assignment step (Algorithm 3, Section 3): for each object x_i, rho <- 0;
 * for each term s of x_i in ascending order and each tuple (c, u) of the
 * means' inverted file xi_s (ascending c): rho_c += v * u; then the first
 * maximum over j = 0..K-1 with a strict '>' (reading: lowest id among the
 * maxima, an all-zero rho goes to cluster 0).  Objects are independent, so
 * the loop over objects is split across OpenMP threads; each thread owns
 * one rho array.  mults counts the multiplications (Eq. 15).
 *
 * Update step (Algorithm 3): per cluster j a dense w in R^D, w_s += v over
 * the members in ascending object id and their terms in ascending order,
 * w_p /= |C_j|, then the tuples (j, w_p / ||w||_2) for w_p != 0 appended to
 * xi_p in ascending j.  An empty cluster (or a zero w) keeps its previous
 * tuples when empty_policy is 0 and gets none when it is 1.  Clusters are
 * independent, so they are split across threads (one w per thread); the
 * term-major lists are assembled afterwards in ascending j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ALG3_OK 0
#define ALG3_E_INVALID 1
#define ALG3_E_OOM 3

static int n_threads_for(int requested) {
#ifdef _OPENMP
  return requested > 0 ? requested : omp_get_max_threads();
#else
  (void)requested;
  return 1;
#endif
}

int alg3_threads_available(void) { return n_threads_for(0); }

/* rows == NULL: every object i < n_docs; otherwise the n_rows listed objects,
 * written to assign[q] / best[q] for q < n_rows. */
int alg3_assign(int64_t n_docs, const int64_t* row_ptr, const int32_t* term, const float* val, int32_t k,
                int64_t n_terms, const int64_t* xi_ptr, const int32_t* xi_c, const double* xi_u,
                const int64_t* rows, int64_t n_rows, int32_t* assign, double* best, int64_t* mults_out,
                int threads) {
  if (k < 1 || n_docs < 0 || !row_ptr || !xi_ptr || !assign || !best) return ALG3_E_INVALID;
  const int64_t n_out = rows ? n_rows : n_docs;
  const int nt = n_threads_for(threads);
  int status = ALG3_OK;
  int64_t mults = 0;
#pragma omp parallel num_threads(nt) reduction(+ : mults)
  {
    double* rho = (double*)malloc(sizeof(double) * (size_t)k);
    if (!rho) {
#pragma omp atomic write
      status = ALG3_E_OOM;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t q = 0; q < n_out; ++q) {
        const int64_t i = rows ? rows[q] : q;
        if (i < 0 || i >= n_docs) {
#pragma omp atomic write
          status = ALG3_E_INVALID;
          continue;
        }
        for (int32_t j = 0; j < k; ++j) rho[j] = 0.0;
        for (int64_t h = row_ptr[i]; h < row_ptr[i + 1]; ++h) {
          const int32_t s = term[h];
          if (s < 0 || (int64_t)s >= n_terms) continue;
          const double v = (double)val[h];
          for (int64_t e = xi_ptr[s]; e < xi_ptr[s + 1]; ++e) {
            const double prod = v * xi_u[e];
            rho[xi_c[e]] = rho[xi_c[e]] + prod;
          }
          mults += xi_ptr[s + 1] - xi_ptr[s];
        }
        double rmax = rho[0];
        int32_t a = 0;
        for (int32_t j = 1; j < k; ++j)
          if (rho[j] > rmax) {
            rmax = rho[j];
            a = j;
          }
        assign[q] = a;
        best[q] = rmax;
      }
      free(rho);
    }
  }
  if (mults_out) *mults_out = mults;
  return status;
}

/* Update step.  Outputs the new inverted file: out_ptr[n_terms + 1] and up to
 * out_cap tuples in out_c / out_u.  Returns ALG3_E_OOM (with *out_len set to
 * the length needed) when out_cap is too small.  prev_* is the inverted file
 * the assignment used (for empty_policy 0).  Only clusters j0 <= j < j1 get
 * rows (the whole update is j0 = 0, j1 = k; a range times a sample of it). */
int alg3_update(int64_t n_docs, const int64_t* row_ptr, const int32_t* term, const float* val, int32_t k,
                int64_t n_terms, const int32_t* assign, const int64_t* prev_ptr, const int32_t* prev_c,
                const double* prev_u, int32_t empty_policy, int32_t j0, int32_t j1, int64_t* out_ptr,
                int32_t* out_c, double* out_u, int64_t out_cap, int64_t* out_len, int threads) {
  if (k < 1 || n_terms < 1 || !assign || !out_ptr || !out_len) return ALG3_E_INVALID;
  if (j0 < 0 || j1 > k || j0 > j1) return ALG3_E_INVALID;
  const int nt = n_threads_for(threads);
  int status = ALG3_OK;
  /* C_j in ascending object id (a stable counting sort of the objects) */
  int64_t* cl_ptr = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  int64_t* members = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_docs > 0 ? n_docs : 1));
  /* previous means cluster-major, for clusters that keep their tuples */
  int64_t* pr_ptr = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  const int64_t e_prev = prev_ptr ? prev_ptr[n_terms] : 0;
  int32_t* pr_t = (int32_t*)malloc(sizeof(int32_t) * (size_t)(e_prev > 0 ? e_prev : 1));
  double* pr_u = (double*)malloc(sizeof(double) * (size_t)(e_prev > 0 ? e_prev : 1));
  /* per-cluster new rows, then term-major */
  int64_t* row_len = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  int32_t** row_t = (int32_t**)calloc((size_t)k, sizeof(int32_t*));
  double** row_u = (double**)calloc((size_t)k, sizeof(double*));
  if (!cl_ptr || !members || !pr_ptr || !pr_t || !pr_u || !row_len || !row_t || !row_u) {
    status = ALG3_E_OOM;
    goto done;
  }
  for (int64_t i = 0; i < n_docs; ++i) {
    if (assign[i] < 0 || assign[i] >= k) {
      status = ALG3_E_INVALID;
      goto done;
    }
    cl_ptr[assign[i] + 1]++;
  }
  for (int32_t j = 0; j < k; ++j) cl_ptr[j + 1] += cl_ptr[j];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    if (!fill) {
      status = ALG3_E_OOM;
      goto done;
    }
    memcpy(fill, cl_ptr, sizeof(int64_t) * (size_t)k);
    for (int64_t i = 0; i < n_docs; ++i) members[fill[assign[i]]++] = i;
    free(fill);
  }
  if (prev_ptr) {
    for (int64_t p = 0; p < n_terms; ++p)
      for (int64_t e = prev_ptr[p]; e < prev_ptr[p + 1]; ++e) pr_ptr[prev_c[e] + 1]++;
    for (int32_t j = 0; j < k; ++j) pr_ptr[j + 1] += pr_ptr[j];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    if (!fill) {
      status = ALG3_E_OOM;
      goto done;
    }
    memcpy(fill, pr_ptr, sizeof(int64_t) * (size_t)k);
    for (int64_t p = 0; p < n_terms; ++p)
      for (int64_t e = prev_ptr[p]; e < prev_ptr[p + 1]; ++e) {
        const int64_t o = fill[prev_c[e]]++;
        pr_t[o] = (int32_t)p;
        pr_u[o] = prev_u[e];
      }
    free(fill);
  }
#pragma omp parallel num_threads(nt)
  {
    double* w = (double*)malloc(sizeof(double) * (size_t)n_terms);
    if (!w) {
#pragma omp atomic write
      status = ALG3_E_OOM;
    } else {
#pragma omp for schedule(dynamic, 4)
      for (int32_t j = j0; j < j1; ++j) {
        for (int64_t p = 0; p < n_terms; ++p) w[p] = 0.0;
        const int64_t size = cl_ptr[j + 1] - cl_ptr[j];
        for (int64_t q = cl_ptr[j]; q < cl_ptr[j + 1]; ++q) {
          const int64_t i = members[q];
          for (int64_t h = row_ptr[i]; h < row_ptr[i + 1]; ++h) w[term[h]] = w[term[h]] + (double)val[h];
        }
        if (size > 0)
          for (int64_t p = 0; p < n_terms; ++p) w[p] = w[p] / (double)size;
        double n2 = 0.0;
        for (int64_t p = 0; p < n_terms; ++p) n2 = n2 + w[p] * w[p];
        const double norm = sqrt(n2);
        if (size == 0 || norm == 0.0) {
          if (empty_policy == 0 && prev_ptr) {
            const int64_t len = pr_ptr[j + 1] - pr_ptr[j];
            row_t[j] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(len > 0 ? len : 1));
            row_u[j] = (double*)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
            if (!row_t[j] || !row_u[j]) {
#pragma omp atomic write
              status = ALG3_E_OOM;
              continue;
            }
            memcpy(row_t[j], pr_t + pr_ptr[j], sizeof(int32_t) * (size_t)len);
            memcpy(row_u[j], pr_u + pr_ptr[j], sizeof(double) * (size_t)len);
            row_len[j] = len;
          }
          continue;
        }
        int64_t len = 0;
        for (int64_t p = 0; p < n_terms; ++p) len += w[p] != 0.0;
        row_t[j] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(len > 0 ? len : 1));
        row_u[j] = (double*)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
        if (!row_t[j] || !row_u[j]) {
#pragma omp atomic write
          status = ALG3_E_OOM;
          continue;
        }
        int64_t o = 0;
        for (int64_t p = 0; p < n_terms; ++p)
          if (w[p] != 0.0) {
            row_t[j][o] = (int32_t)p;
            row_u[j][o] = w[p] / norm;
            ++o;
          }
        row_len[j] = len;
      }
      free(w);
    }
  }
  if (status != ALG3_OK) goto done;
  {
    int64_t total = 0;
    for (int32_t j = 0; j < k; ++j) total += row_len[j];
    *out_len = total;
    if (total > out_cap || !out_c || !out_u) {
      status = ALG3_E_OOM;
      goto done;
    }
    for (int64_t p = 0; p <= n_terms; ++p) out_ptr[p] = 0;
    for (int32_t j = 0; j < k; ++j)
      for (int64_t q = 0; q < row_len[j]; ++q) out_ptr[row_t[j][q] + 1]++;
    for (int64_t p = 0; p < n_terms; ++p) out_ptr[p + 1] += out_ptr[p];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_terms);
    if (!fill) {
      status = ALG3_E_OOM;
      goto done;
    }
    memcpy(fill, out_ptr, sizeof(int64_t) * (size_t)n_terms);
    for (int32_t j = 0; j < k; ++j) /* ascending j: every list ends up ascending in c */
      for (int64_t q = 0; q < row_len[j]; ++q) {
        const int64_t o = fill[row_t[j][q]]++;
        out_c[o] = j;
        out_u[o] = row_u[j][q];
      }
    free(fill);
  }
done:
  if (row_t)
    for (int32_t j = 0; j < k; ++j) free(row_t[j]);
  if (row_u)
    for (int32_t j = 0; j < k; ++j) free(row_u[j]);
  free(row_t);
  free(row_u);
  free(row_len);
  free(pr_t);
  free(pr_u);
  free(pr_ptr);
  free(members);
  free(cl_ptr);
  return status;
}
