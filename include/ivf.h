/*
 * ivf.h -- C ABI of libivfkm: inverted-file spherical k-means (IVF) on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method is the Lloyd iteration of Aoyama, Saito and Ikeda,
 * "Inverted-File k-Means Clustering: Performance Analysis" (arXiv 2002.09094):
 *   - problem: spherical k-means, Section 2.2, Eqs. 4-5, Algorithm 2 -- N
 *     unit-L2 sparse objects, K unit-L2 means, maximise the summed cosine
 *     similarity;
 *   - data structures: objects in the standard sparse expression (Section
 *     2.3, Fig. 1(a)) = CSR rows of (term id, value) sorted by term id; means
 *     in the inverted-file expression (Section 3) = for every term s the list
 *     xi_s of (cluster id c, value u) in ascending c;
 *   - one iteration (Algorithm 3): the assignment step scatters
 *     rho_c += v * u over the posting lists of the object's terms and takes
 *     the argmax; the update step sums each cluster's members, normalises,
 *     and rebuilds the inverted file.
 *
 * Conventions (all calls):
 *   - Ids are 0-based (the paper counts from 1).
 *   - Input arrays may be host or device pointers (the library copies them
 *     with cudaMemcpyDefault); the library keeps no caller pointer after a
 *     call returns, except that ivf_load_objects reads its sources until the
 *     next ivf_assign / ivf_iterate / ivf_set_means_from_docs returns.
 *     Output arrays of ivf_assign are DEVICE pointers (or NULL); the
 *     ivf_get_* calls write to host or device pointers.
 *   - Every call is ordered on the CUDA stream given at create time and
 *     returns after enqueueing, except where a comment says it synchronises
 *     (ivf_load_objects copies on a second stream of the context, ordered
 *     with the first as its comment says).
 *   - Errors come back as an ivf_status; the library never aborts or traps.
 *     After IVF_E_INVALID or IVF_E_STATE the context is unchanged and still
 *     usable; after IVF_E_CUDA destroy it.  ivf_last_error() gives a message.
 *   - Ties in the argmax go to the lowest cluster id (an object that shares
 *     no term with any mean therefore goes to cluster 0).  An empty cluster
 *     keeps its previous mean (empty_policy 0) or gets an empty mean
 *     (empty_policy 1).  A mean element that sums to exactly 0 is dropped,
 *     as Algorithm 3's "w_p != 0" test does.
 */
#ifndef IVFKM_IVF_H
#define IVFKM_IVF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ivf_ctx ivf_ctx; /* opaque, owned by the library */

typedef enum {
  IVF_OK = 0,
  IVF_E_INVALID = 1,     /* bad argument or malformed input; nothing changed */
  IVF_E_STATE = 2,       /* call out of order (e.g. assign before set_means) */
  IVF_E_OOM = 3,         /* device allocation failed or a capacity was exceeded */
  IVF_E_CUDA = 4,        /* a CUDA call failed; destroy the context */
  IVF_E_TIMEOUT = 5,     /* a bounded device wait ran out */
  IVF_E_UNSUPPORTED = 6  /* valid request the library does not handle */
} ivf_status;

/* Storage type of the object and mean values streamed by the assignment
 * step.  Accumulation is FP32 in every case; FP32 master copies of the
 * object values and FP64 master means are kept for the update step and the
 * FP64 re-score. */
typedef enum { IVF_F32 = 0, IVF_F16 = 1, IVF_BF16 = 2 } ivf_dtype;

/* ivf_config.flags */
#define IVF_FLAG_VALIDATE 1u  /* check CSR rows (sorted, unique, in range, finite) at create/load */
#define IVF_FLAG_NO_GRAPH 2u  /* ivf_iterate launches kernels directly instead of a CUDA graph */
#define IVF_FLAG_DENSE_HEAD 4u  /* autotune only among CUDA-core dense-head kernels: posting lists that cover
                                   at least a fraction theta of the K clusters are also stored as
                                   dense rows (the paper's full inverted file, IFN, Section 4,
                                   for those terms only) and accumulated in registers */
#define IVF_FLAG_SPARSE_ONLY 8u /* autotune only among kernels that read the sparse lists alone */
#define IVF_FLAG_TENSOR_HEAD 16u /* FP16/BF16 storage: autotune only among dense-head kernels whose
                                    head part is a tensor-core GEMM of the objects' dense head
                                    values with the dense rows (the library's tcgen05 kernel),
                                    batch by batch */
#define IVF_FLAG_TILE_MAJOR 32u  /* autotune only among tile-major schedules: one launch per tile of the
                                    cluster range over all objects, (best, id, second) carried in
                                    device memory between launches (tiled shapes, one instance) */
#define IVF_FLAG_OBJECT_MAJOR 64u /* autotune only among object-major schedules (each object walks all
                                     of its cluster tiles in one launch) */
#define IVF_FLAG_IVFD 128u  /* the paper's comparison algorithm IVFD (Algorithm 4, Section 7.2) instead
                               of IVF for the assignment step: the objects are also held as an
                               inverted file (term-major (object, value) lists, built once per object
                               set) and the assignment loops over the means, each mean's terms
                               scattering into per-object accumulators.  Same multiplications
                               (Eq. 15) and, for FP32, the same similarity bits as IVF's sparse
                               kernel; near-ties are re-scored in FP64 against every cluster.  FP32
                               storage, one instance (else IVF_E_UNSUPPORTED).  The update step is
                               IVF's (the paper's IVFD also updates from the standard sparse form). */

typedef struct {
  int64_t n_docs;      /* N >= 1 */
  int64_t n_terms;     /* D >= 1 */
  int64_t nnz;         /* number of (term, value) tuples over all objects */
  int32_t k;           /* number of clusters, 1 <= k <= N */
  int32_t storage;     /* ivf_dtype */
  int32_t rescore;     /* 1: FP64 re-score of objects whose top-2 gap is within the
                          computed error bound (default and required for exact
                          assignments); 0: off */
  int32_t empty_policy;/* 0 keep previous mean (default), 1 empty mean */
  int32_t k_tile;      /* accumulator tile over the cluster range: 0 = autotune,
                          else a power of two in [512, 65536] or >= k (no tiling);
                          with IVF_FLAG_DENSE_HEAD it fixes the dense-head kernel's
                          shared-memory tile (512: 512-cluster head tile; 1024 and
                          more: k_tile / 1024 head tiles of 1,024 clusters), with
                          IVF_FLAG_TENSOR_HEAD the same for the tensor-core head
                          (a multiple of 1024; theta 0.25) */
  int32_t warps_per_block; /* 0 = autotune, else 1..32 */
  uint32_t flags;      /* IVF_FLAG_* */
  int32_t means_capacity; /* entries reserved for the means / inverted file at create
                             (0 = automatic); the arrays grow on demand */
  int64_t dense_head_bytes; /* device memory first reserved for dense head rows
                               (0 = 2 GiB); grows on demand up to 24 GiB when more
                               lists qualify (the lists that do not fit are read
                               from the sparse inverted file: exact, slower) */
} ivf_config;

/* Per-iteration statistics (Section 5.2 reports time and memory per
 * iteration; Eq. 15 counts the multiplications). */
typedef struct {
  int64_t n_changed;       /* objects whose assignment differs from the previous one
                              (all N on the first assignment) */
  int64_t entries_visited; /* posting entries multiplied: sum_i sum_h (nc)_{t_(i,h)}, Eq. 15 */
  int64_t ivf_entries;     /* E = sum_p (nc)_p, tuples in the inverted file used */
  int64_t n_zero_sim;      /* objects that share no term with any mean (they meet no posting
                              entry; Algorithm 3 never assigns them, here they go to cluster 0) */
  int64_t n_flagged;       /* objects whose FP32 top-2 gap was within the error bound */
  int64_t n_rescored;      /* objects re-scored in FP64 */
  double objective;        /* J = sum_i rho(x_i, mu_a(i)), Eq. 5, FP64 accumulation */
  float t_assign_ms;       /* device time of the last assignment step (0 if not timed) */
  float t_update_ms;       /* device time of the last update step (0 if not timed) */
} ivf_iter_stats;

typedef struct {
  int64_t n_docs, n_terms, nnz;
  int32_t k, n_instances;
  int64_t ivf_entries;     /* E of the current means */
  int64_t ivf_capacity;    /* maximum E the context can hold */
  int32_t k_tile, warps_per_block; /* launch shape in use (after autotune) */
  int32_t iteration;       /* completed update steps */
  int32_t storage;
  int64_t device_bytes;    /* device memory held by the context */
  int32_t dense_head_r;    /* 0: sparse kernel; else dense-head kernel with 32*r-cluster head tiles */
  int32_t dense_head_sub;  /* head tiles per shared-memory tile of the dense-head kernel */
  int32_t dense_head_tensor; /* 1: the head part is computed by a tensor-core GEMM */
  float dense_head_theta;  /* lists covering >= theta * K clusters are stored densely */
  int64_t dense_head_rows; /* dense rows in the inverted file last built */
  int32_t tile_major;      /* 1: the assignment runs tile-major (one launch per cluster tile) */
} ivf_info;

/* Create a context for one clustering problem and copy the objects in.
 * row_ptr: int64[N+1], row_ptr[0] = 0, row_ptr[N] = nnz, non-decreasing.
 * term: int32[nnz], ascending and unique inside each row, in [0, D).
 * val: float[nnz], finite; each row is expected to have unit L2 norm
 *      (Section 2.2: objects are points on the unit hypersphere).
 * cuda_stream: cudaStream_t for all work of the context (NULL = legacy default).
 * On success *out holds the context; on error *out is NULL. */
ivf_status ivf_create(const ivf_config* cfg, const int64_t* row_ptr, const int32_t* term,
                      const float* val, void* cuda_stream, ivf_ctx** out);

/* Replace the object values and terms (same N and nnz as at create time):
 * the host->device copy of a new batch of objects.  Row structure may
 * change.  Means and assignments are kept.
 * The copy goes to a staging buffer on a second stream of the context, so it
 * can run while work already on the context stream (an assignment) computes.
 * The new objects take effect, in stream order, at the next ivf_assign,
 * ivf_iterate or ivf_set_means_from_docs; ivf_update keeps working on the
 * objects its assignment ran on.  Device sources are read after the work
 * already on the context stream; host sources (pinned or pageable) are read
 * asynchronously and must stay unchanged until one of those three calls (or
 * ivf_destroy) returns.  A second load before then replaces the first.
 * row_ptr is checked on the device (starts at 0, ends at nnz, non-decreasing)
 * before the term and value copies are issued, which synchronises the copy
 * stream once; on IVF_E_INVALID the current objects stay in place.  With
 * IVF_FLAG_VALIDATE the rows are also checked as at create time. */
ivf_status ivf_load_objects(ivf_ctx* ctx, const int64_t* row_ptr, const int32_t* term,
                            const float* val);

/* Set the K means from cluster-major sparse rows (mean j = row j):
 * mean_ptr int64[K+1], mean_term int32[E0] ascending and unique per row,
 * mean_val float[E0].  Each row is divided by its FP64 L2 norm (Algorithm
 * 2's normalisation); a row of zero norm is IVF_E_INVALID.  The inverted
 * file (Section 3) is built from the result.  Resets the iteration count and
 * forgets previous assignments. */
ivf_status ivf_set_means(ivf_ctx* ctx, const int64_t* mean_ptr, const int32_t* mean_term,
                         const float* mean_val);

/* Initial means from K distinct objects: mean j = x_{doc_ids[j]} / ||x||
 * (Section 5.3: the initial state is chosen at random).  doc_ids: int32[K]. */
ivf_status ivf_set_means_from_docs(ivf_ctx* ctx, const int32_t* doc_ids);

/* Assignment step of Algorithm 3 (the triple loop and the argmax) for all
 * objects against the current means, then the FP64 re-score of near-ties
 * and the reductions for the statistics.
 * assign_out: device int32[N] or NULL; best_out: device float[N] or NULL
 * (rho of the chosen cluster); gap_out: device float[N] or NULL (best minus
 * second best).  The results also stay in the context for ivf_update.
 * stats_out: host pointer or NULL; when given, the call synchronises the
 * stream and fills it. */
ivf_status ivf_assign(ivf_ctx* ctx, int32_t* assign_out, float* best_out, float* gap_out,
                      ivf_iter_stats* stats_out);

/* Update step of Algorithm 3 from the last assignment: member sums in FP64,
 * L2 normalisation, inverted-file rebuild.  Synchronises the stream once to
 * check that the new means fit; if not, it grows the arrays and redoes the
 * step (IVF_E_OOM if the device has no room). */
ivf_status ivf_update(ivf_ctx* ctx);

/* Data-parallel update over object shards (one context per rank, each
 * holding a contiguous shard of the objects and the same means).  The
 * update of Algorithm 3 sums each cluster's members; split by shard,
 *   s_j = sum over shards r of s_j^(r),  s_j^(r) = sum_{i in C_j, i in shard r} x_i,
 * so each rank computes its own member sums, the ranks exchange them, and
 * every rank finishes the same update from all of them.
 *
 * ivf_get_partial_sums: this context's member sums for its last assignment
 * (the first half of the update step), before normalisation.  *n_out (host)
 * receives U, the number of (cluster, term) pairs its members touch; when
 * any of cluster / term / sum is given (host or device, capacity cap >= U,
 * else IVF_E_INVALID), they receive cluster int32[U] (cluster ids), term
 * int32[U] and sum double[U] (FP64, members in ascending object id), in
 * ascending (cluster, term).  A sum can be exactly 0 (values of both signs).
 * One-instance contexts only.  Synchronises the stream. */
ivf_status ivf_get_partial_sums(ivf_ctx* ctx, int64_t cap, int32_t* cluster, int32_t* term, double* sum,
                                int64_t* n_out);
/* ivf_update_from_partials: the update step from member sums gathered from
 * every shard -- the shards' lists as ivf_get_partial_sums returns them,
 * concatenated in shard order (n_total entries; host or device arrays,
 * copied in).  Equal (cluster, term) pairs are added in FP64 in the order
 * given (shard order), so every rank that passes the same lists gets the
 * same bits; then, as ivf_update: normalisation, the empty-cluster policy
 * (from this context's current means), and the inverted-file rebuild.  An
 * id outside [0, k) or [0, n_terms) is IVF_E_INVALID before any change.
 * Synchronises the stream.  The sums of one shard alone give ivf_update's
 * means exactly; with several shards, each sum is the shards' partial sums
 * added in shard order (FP64 reassociated against the one-context order,
 * about 1e-16 relative). */
ivf_status ivf_update_from_partials(ivf_ctx* ctx, int64_t n_total, const int32_t* cluster, const int32_t* term,
                                    const double* sum);

/* Run assignment + update until no assignment changes (from the second
 * iteration on) or max_iter iterations.  Synchronises once per iteration to
 * read the change count.  iters_done / converged / last_stats may be NULL. */
ivf_status ivf_iterate(ivf_ctx* ctx, int32_t max_iter, int32_t* iters_done, int32_t* converged,
                       ivf_iter_stats* last_stats);

/* Copies out (host or device destination; these synchronise the stream). */
ivf_status ivf_get_assign(ivf_ctx* ctx, int32_t* out);        /* int32[N] */
ivf_status ivf_get_best(ivf_ctx* ctx, float* out);            /* float[N] */
ivf_status ivf_get_gap(ivf_ctx* ctx, float* out);             /* float[N] */
/* Per-result error statement of the last assignment: out[i] >= |best_i - rho_i|
 * where best_i is the returned best similarity and rho_i the exact similarity
 * of object i to its returned cluster under the FP64 master means.  For an
 * object scored in FP32 accumulation it is the bound E_i that decides the
 * re-score (FP32 storage: mean rounding plus FMA recursive summation over the
 * object's m terms; FP16/BF16: both operands' rounding, the FP16 subnormal
 * floor and the same summation term; relative to best_i when every object
 * and mean value is >= 0, else scaled by ||x_i||); for an object re-scored
 * in FP64 it is the FP64 summation error plus the rounding of best_i to
 * float; 0 for an object that met no posting entry.  float[N]. */
ivf_status ivf_get_err_bound(ivf_ctx* ctx, float* out);
ivf_status ivf_get_info(ivf_ctx* ctx, ivf_info* out);         /* host */
/* FP64 master means, cluster-major: ptr int64[K+1], term int32[E], val double[E];
 * any of the three may be NULL. */
ivf_status ivf_get_means(ivf_ctx* ctx, int64_t* ptr, int32_t* term, double* val);
/* The inverted file as streamed by the assignment: term_ptr int64[D+1],
 * cid int32[E] (cluster ids), w float[E] (values after the storage cast,
 * widened to float); any may be NULL. */
ivf_status ivf_get_inverted_file(ivf_ctx* ctx, int64_t* term_ptr, int32_t* cid, float* w);
/* Clusters C_j of the last update: cl_ptr int64[K+1], members int32[N] in
 * ascending object id inside each cluster; either may be NULL. */
ivf_status ivf_get_members(ivf_ctx* ctx, int64_t* cl_ptr, int32_t* members);
/* Set the "previous" assignment used for n_changed (checkpoint resume). */
ivf_status ivf_set_assign(ivf_ctx* ctx, const int32_t* assign);
/* Restore FP64 master means exactly (checkpoint resume), cluster-major as
 * returned by ivf_get_means; no renormalisation. */
ivf_status ivf_restore_means(ivf_ctx* ctx, const int64_t* ptr, const int32_t* term,
                             const double* val, int32_t iteration);

/* Message of the last error on this context (never NULL). */
const char* ivf_last_error(const ivf_ctx* ctx);
/* Frees everything the context holds.  NULL is a no-op. */
void ivf_destroy(ivf_ctx* ctx);

/* Device-time accounting over a window of calls (Section 5.2 measures CPU
 * time per iteration; this is its GPU counterpart).  While enabled, every
 * ivf_assign / ivf_update call records CUDA events on the context stream
 * around its kernels; nothing synchronises until ivf_get_timing. */
typedef struct {
  int32_t n_assign;         /* ivf_assign calls in the window */
  int32_t n_update;         /* ivf_update calls in the window */
  double assign_kernel_ms;  /* sum: the assignment kernel alone (with the tensor-core head:
                               the dense head values, the GEMM and the kernel, batch by batch;
                               with a batched context: the launches of every class) */
  double assign_step_ms;    /* sum: assignment kernel + FP64 re-score + reductions */
  double update_ms;         /* sum: update step including the inverted-file rebuild */
  int64_t entries_visited;  /* sum of the Eq. 15 multiplication counts */
  int64_t n_rescored;       /* sum of objects re-scored in FP64 */
} ivf_timing;
/* Start a new window (enable = 1) or stop recording (enable = 0). */
ivf_status ivf_timing_reset(ivf_ctx* ctx, int32_t enable);
/* Sums over the window so far; synchronises the stream. */
ivf_status ivf_get_timing(ivf_ctx* ctx, ivf_timing* out);

/* The tensor-core block of the dense head (the paper's full inverted file
 * IFN, Section 4, for the terms whose posting lists are dense), on caller
 * buffers: d[i][c] = sum_{s < k} a[i][s] * b[c][s] for i < m, c < n, with a
 * (m x k), b (n x k) and d (m x n) row-major DEVICE matrices of 16-bit
 * values (storage IVF_F16 or IVF_BF16, all three the same type), leading
 * dimensions lda, ldb, ldd in elements (multiples of 8, pointers 16-byte
 * aligned), FP32 accumulation on the tensor cores (tcgen05, operands staged
 * by TMA), d rounded to the 16-bit type.  n must be a multiple of 256 and k
 * of 64 (IVF_E_INVALID otherwise).  This is the kernel the FP16/BF16
 * assignment uses for its head part, batch by batch.  Synchronises the
 * stream; IVF_E_TIMEOUT if a bounded device wait ran out. */
ivf_status ivf_head_product(int64_t m, int32_t n, int32_t k, const void* a, int64_t lda, const void* b,
                            int64_t ldb, void* d, int64_t ldd, int32_t storage, void* cuda_stream);

/* Platform probe (no counterpart in the paper): the read bandwidth, in GB/s,
 * that the current device delivers from a resident set of `bytes` bytes
 * (>= 1 MiB, a multiple of 16, small enough to stay in L2) read `reps` times
 * per launch with 16-byte L2-only loads by 4 blocks of 512 threads per SM;
 * the best of five launches after one warm-up.  The assignment kernel's
 * posting reads are served mostly by L2, so its bytes per second are
 * reported against this figure.  Allocates and frees its own buffer;
 * synchronises the stream. */
ivf_status ivf_probe_l2_read(int64_t bytes, int32_t reps, void* cuda_stream, double* gbs_out);

/* Number of kernels this library has launched in the process so far (all
 * of them its own, the tensor-core head product included). */
int64_t ivf_launch_count(void);
/* Library version string. */
const char* ivf_version(void);

/* ------------------------------------------------------------------------
 * Batched form: many independent clustering problems of uneven N, K and D
 * in one context.  Every launch (re-score, update) covers all instances at
 * once, and the assignment one launch per class of instances by K (<= 128,
 * <= 256, <= 512, <= 1,024, <= 1,536, <= 2,048, larger), each with its own
 * autotuned kernel; no arithmetic mixes instances.
 * inst_docs int64[n_inst+1]: object offsets (row_ptr is the concatenation of
 *   the instances' CSR rows, term ids local to the instance);
 * inst_terms int32[n_inst]: D of each instance; inst_k int32[n_inst]: K.
 * cfg supplies storage, rescore, empty_policy, k_tile, warps, flags;
 * cfg->n_docs/n_terms/nnz/k are ignored (taken from the arrays).
 * Means: ivf_set_means_from_docs with doc_ids int32[sum K] holding each
 * instance's K local document ids in instance order.  ivf_get_assign
 * returns local cluster ids. ------------------------------------------- */
ivf_status ivfb_create(const ivf_config* cfg, int32_t n_inst, const int64_t* inst_docs,
                       const int32_t* inst_terms, const int32_t* inst_k, const int64_t* row_ptr,
                       const int32_t* term, const float* val, void* cuda_stream, ivf_ctx** out);
/* Per-instance change counts of the last assignment: int64[n_inst] (host or device). */
ivf_status ivfb_get_changed(ivf_ctx* ctx, int64_t* out);

/* ------------------------------------------------------------------------
 * Allocation-free assignment step.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory where they run
 * the assignment -- applications whose device memory is owned by their own
 * pool or framework allocator, latency-critical loops that must not pay for
 * (or synchronise the device on) a cudaMalloc after start-up, and services
 * that reserve all memory once.  It allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine, and no context.
 *
 * The caller passes every input and output as DEVICE pointers:
 *   objects: row_ptr int64[N+1], term int32[nnz], val float[nnz] (CSR, as
 *     for ivf_create).  They are read only and NOT validated: row_ptr must
 *     start at 0 and not decrease, terms must be ascending, unique and in
 *     [0, n_terms) in each row, and values finite; rows that break this give
 *     undefined results (a term id out of range is read out of bounds);
 *   the inverted file of the means: term_ptr int64[D+1], cid int32[E]
 *     (cluster ids, ascending inside each term's list), w float[E];
 *   the FP64 means it was cast from, cluster-major: mean_ptr int64[K+1],
 *     mean_term int32[E], mean_val double[E] (ivf_get_inverted_file and
 *     ivf_get_means return exactly these);
 *   outputs: assign_out int32[N], best_out float[N] or NULL, gap_out float[N]
 *     or NULL.
 * The result equals ivf_assign's on a context with FP32 storage and
 * rescore = 1: the FP64 argmax (lowest cluster id on ties), the FP32 best
 * similarity, and the top-2 gap.
 *
 * The call's scratch -- work counters, object norms, and the queue of
 * near-tie objects for the FP64 re-score -- lives in one file-scope static
 * device array of IVF_STATIC_SCRATCH_BYTES bytes; every GPU that loads this
 * library holds it until the process exits.  Sizes beyond the limits
 * (N > IVF_STATIC_MAX_DOCS, K > IVF_STATIC_MAX_K, K > N) return
 * IVF_E_INVALID before any GPU work; a failing CUDA call returns IVF_E_CUDA.
 * The first call on a device does a one-time set-up there (it looks up the
 * scratch array's device address with cudaGetSymbolAddress and raises the
 * kernel's shared-memory limit); make that first call before any stream
 * capture.  All calls share the one array, which keeps the last call's
 * contents (each call clears what must start at zero): calls that overlap
 * on the GPU -- from two streams or two threads -- race, so the caller must
 * serialise them.  The call returns after enqueueing its kernels on
 * cuda_stream. */
#define IVF_STATIC_MAX_DOCS 16384
#define IVF_STATIC_MAX_K 12288
#define IVF_STATIC_SCRATCH_BYTES 2425088
ivf_status ivf_assign_static(int64_t n_docs, const int64_t* row_ptr, const int32_t* term, const float* val,
                             int64_t n_terms, int32_t k, const int64_t* term_ptr, const int32_t* cid,
                             const float* w, const int64_t* mean_ptr, const int32_t* mean_term,
                             const double* mean_val, int32_t* assign_out, float* best_out, float* gap_out,
                             void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* IVFKM_IVF_H */
