// Internal launch interface between the C ABI (ivf_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ivfk {

enum Storage : int { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

// Candidate clusters kept per flagged object for the FP64 re-score (more
// candidates, or a flagged object beyond the slots of the candidate slab,
// means a re-score against every cluster).
constexpr int CAND_MAX = 128;

// Device status word bits (ctx->d_status).
enum StatusBits : unsigned {
  STS_CAPACITY = 1u,   // the new means did not fit the inverted-file capacity
  STS_BAD_MEANS = 2u,  // a mean row given by the caller has zero norm or bad terms
  STS_BAD_ROWS = 4u,   // object rows failed validation
  STS_TIMEOUT = 8u,    // a bounded device wait ran out
};

// Everything the assignment kernel reads and writes.
struct AssignArgs {
  int64_t n_docs;          // work items: objects 0, s, 2s, ... (s = obj_stride) below n_docs * s
  int32_t obj_stride = 1;  // 1 except when the autotuner times a strided sample
  const int64_t* row_ptr;  // [N+1]
  const int32_t* term;     // [nnz] global term ids
  const void* val;         // [nnz] storage type
  const float* nx;         // [N] object norm, rounded up
  int32_t n_inst;
  const int64_t* inst_docs;  // [n_inst+1]
  const int32_t* inst_clu;   // [n_inst+1]
  // Optional subset of the instances (a batched context launches one kernel
  // per class of instances): work item o belongs to listed instance q with
  // obj_prefix[q] <= o < obj_prefix[q+1]; null = every object in order.
  const int32_t* obj_inst;   // [n_obj_inst]
  const int64_t* obj_prefix; // [n_obj_inst+1]
  int32_t n_obj_inst;
  const int64_t* term_ptr;   // [D+1]
  const void* cid;           // [E] local cluster id & 0xFFFF (uint16), or int32 ids
  const void* w;             // [E] storage type
  const int32_t* toff;       // [D * (n_tiles_max+1)] per (term, tile) offset inside the list, or null
  int32_t n_tiles_max;
  int32_t k_tile;            // clusters per tile (power of two when tiled)
  int32_t tiled;
  int32_t tile_cap;          // floats of accumulator per warp (multiple of 4)
  int32_t storage;
  int32_t rescore;
  int32_t* assign;           // [N]
  float* best;               // [N]
  float* gap;                // [N]
  float* err = nullptr;      // [N] or null: bound on |best - rho_FP64| of the returned best
  unsigned long long* work;     // object counter, zero before launch
  unsigned long long* entries;  // visited posting entries (accumulated)
  unsigned long long* n_zero_sim = nullptr;  // objects that met no posting entry (accumulated), or null
  unsigned int* n_flagged;      // flagged objects (accumulated from 0)
  int32_t* flag_obj;            // [N]
  int32_t* flag_cnt;            // [N] candidates, -1 = overflow (all clusters)
  int32_t* flag_cand;           // [cand_slots * CAND_MAX]
  int64_t cand_slots;           // flagged objects that get a candidate list
  // The relative error bound for non-negative data applies when nonneg != 0
  // and neither device flag (some object value < 0, some mean value < 0) is set.
  int32_t nonneg;
  const unsigned* negative;        // objects, or null
  const unsigned* means_negative;  // the means the inverted file was built from, or null
  // Dense head rows (the IFN form for the densest posting lists): term t with
  // head_slot[t] >= 0 is read from wd[head_slot[t] * kpad + cluster] instead
  // of its sparse list.  Used by the register-accumulator kernels (head_r > 0).
  const int32_t* head_slot;     // [D] or null
  const void* wd;               // [T * kpad] storage type
  int64_t kpad;                 // row length, a multiple of the head sub-tile (32 * head_r)
  int32_t head_sub = 1;         // head sub-tiles of 32 * head_r clusters per shared-memory tile
  // Tensor-core head (16-bit storage): the head part of rho for objects
  // obj_base + o was computed beforehand by a GEMM of the objects' dense head
  // values with the dense rows (FP32 accumulation, stored as FP16 whatever
  // the storage type: 2^-11 relative rounding, |rho| <= ||x|| far below the
  // FP16 range), rho_head[o * rho_ld + cluster]; the kernel reads it instead
  // of walking the rows.
  const void* rho_head;
  int64_t rho_ld;
  int64_t obj_base;
  // Tile-major schedule: this launch covers the accumulator tiles
  // [tile_lo, tile_hi) of every object (tile_hi = INT_MAX: to the last).  An
  // object whose tiles end inside the range is finished here (gap, error
  // bound, zero-similarity count, near-tie test); otherwise (best, id,
  // second) are carried to the next launch in best / assign / gap.  With
  // tile_lo > 0 the carry of the previous launch is read first.  A finished
  // near-tie is not re-scored here: it is appended to preflag (count in
  // *n_preflag) for an object-major pass that collects its candidates.
  int32_t tile_lo = 0;
  int32_t tile_hi = 0x7fffffff;
  int32_t* preflag = nullptr;
  unsigned int* n_preflag = nullptr;
  // Tile-major candidate carry: each object's candidate clusters for the
  // FP64 re-score collected so far (ids and FP32 values, at most tcand_cap;
  // count -1 = more), so a near-tie needs no second pass unless its list
  // overflowed.  Null = not kept (every near-tie goes to preflag).
  int32_t* tcand = nullptr;   // [N x tcand_cap]
  float* tcandv = nullptr;    // [N x tcand_cap]
  int32_t* tcand_n = nullptr; // [N]
  int32_t tcand_cap = 0;
  // Object-major pass over a list of objects (the near-ties of a tile-major
  // sweep): work item o is object obj_list[o], o < *obj_list_n.
  const int32_t* obj_list = nullptr;
  const unsigned int* obj_list_n = nullptr;
};

// Registers per lane of the head accumulator; the tile is 32 * R clusters.
constexpr int HEAD_R_SMALL = 8;
constexpr int HEAD_R_MID = 16;
constexpr int HEAD_R_LARGE = 32;
constexpr int HEAD_MAX_WARPS = 8;  // warps per block of the dense-head kernels

size_t assign_smem_bytes(int tile_cap, int warps);
cudaError_t assign_prepare(int storage, int tile_cap, int warps, int head_r = 0, int head_sub = 1, bool tc = false);
// head_sub > 1 (split dense-head kernel) is available for head_r == HEAD_R_LARGE and HEAD_R_MID.
cudaError_t launch_assign(const AssignArgs& a, int warps, int blocks, cudaStream_t s, int head_r = 0);
int assign_max_blocks_per_sm(int storage, int tile_cap, int warps, int head_r = 0, int head_sub = 1,
                             bool tc = false);
// FP32 storage, untiled, int32 cluster ids (the caller-held inverted file of ivf_assign_static).
cudaError_t assign_prepare_i32ids(int tile_cap, int warps);
int assign_max_blocks_per_sm_i32ids(int tile_cap, int warps);
cudaError_t launch_assign_i32ids(const AssignArgs& a, int warps, int blocks, cudaStream_t s);

struct RescoreArgs {
  const int64_t* row_ptr;
  const int32_t* term;
  const float* val32;
  int32_t n_inst;
  const int64_t* inst_docs;
  const int32_t* inst_clu;
  const int64_t* mptr;   // [Kt+1] cluster-major FP64 means
  const int32_t* mterm;  // global term ids
  const double* mval;
  const unsigned int* n_flagged;
  const int32_t* flag_obj;
  const int32_t* flag_cnt;
  const int32_t* flag_cand;
  int32_t* assign;
  float* best;
  float* gap;
  float* err;            // [N] or null: bound of the re-scored best
  const float* nx;       // [N] object norms, rounded up (needed with err)
  unsigned long long* n_rescored;
};
cudaError_t launch_rescore(const RescoreArgs& a, int blocks, cudaStream_t s);

struct ReduceArgs {
  int64_t n_docs;
  const int32_t* assign;
  const int32_t* prev;   // null on the first assignment
  const float* best;
  int32_t n_inst;
  const int64_t* inst_docs;
  long long* inst_changed;  // [n_inst], zeroed before launch
  double* part_obj;         // [blocks]
  unsigned long long* part_cnt;  // [2 * blocks]: changed, zero-sim
  double* out_obj;          // [1]
  unsigned long long* out_cnt;   // [2]
  const unsigned long long* zero_sim;  // objects that met no posting entry (from the assignment)
  // window accumulators (added to by the final reduction)
  const unsigned long long* entries;
  const unsigned long long* n_rescored;
  unsigned long long* acc_entries;
  unsigned long long* acc_rescored;
};
cudaError_t launch_reduce(const ReduceArgs& a, int blocks, cudaStream_t s);

// ---------------------------------------------------------------- update
struct UpdateArgs {
  int64_t n_docs, nnz;
  int32_t n_inst;
  int64_t kt;   // total clusters
  int64_t dt;   // total terms
  int tbits, kbits;  // key bits: the largest instance's term count, the total cluster count
  const int64_t* row_ptr;
  const int32_t* term;
  const float* val32;
  const int64_t* inst_docs;
  const int32_t* inst_clu;
  const int64_t* inst_toff;  // [n_inst+1] first global term id of each instance
  const int32_t* assign;  // local cluster ids
  // the objects' tuples in term-major order (zeta): term, and (object << 32
  // | FP32 value bits) of each, ascending object inside each term
  const uint32_t* zterm;
  const uint64_t* zov;
  int32_t empty_policy;
  // old and new cluster-major means
  const int64_t* mptr_old;
  const int32_t* mterm_old;
  const double* mval_old;
  int64_t* mptr_new;
  int32_t* mterm_new;
  double* mval_new;
  int32_t* mclu_new;
  int64_t cap;  // capacity of the means / inverted file arrays
  // members (C_j)
  int64_t* cl_ptr;      // [Kt+1]
  int32_t* members;     // [N]
  double* sum_norm;     // [Kt]
  double* rnorm;        // [Kt] 1 / ||s_j|| rounded to nearest (0 when ||s_j|| = 0)
  // scratch
  uint64_t* k64a;
  uint64_t* k64b;
  uint32_t* v32a;
  uint32_t* v32b;
  uint32_t* flags;      // [nnz+1]
  uint32_t* starts;     // [nnz+1]
  uint64_t* ukey;       // [nnz]
  double* usum;         // [nnz]
  int64_t* uptr;        // [Kt+1]
  int64_t* newlen;      // [Kt+1]
  int32_t* zrun;        // [Kt] 1 when one of cluster j's run sums is exactly zero
  int64_t* d_nnz;       // device copy of nnz
  int64_t* d_n;         // device copy of N
  int64_t* d_u;         // number of unique (cluster, term) keys
  void* temp;           // radix / scan scratch
  unsigned* status;
  unsigned* means_negative;  // set when a written mean value is negative (zeroed by the caller)
};
// The whole update step: members, member sums, new means.
cudaError_t launch_update_means(const UpdateArgs& a, cudaStream_t s);
// Members and member sums (ukey, usum, *d_u) only.
cudaError_t launch_member_sums(const UpdateArgs& a, cudaStream_t s);
// The new means from the run sums (ukey, usum, *d_u <= u_max); a.flags and
// a.starts must hold u_max + 1 entries, ukey / usum u_max.
cudaError_t launch_means_from_sums(const UpdateArgs& a, int64_t u_max, cudaStream_t s);
// Member sums out of (ukey, usum, *d_u): local cluster, term, FP64 sum.
cudaError_t launch_partial_out(const UpdateArgs& a, int64_t u_max, int32_t* cluster, int32_t* term, double* sum,
                               cudaStream_t s);
// Member sums gathered from shards (one instance): (cluster, term, sum)
// lists concatenated in shard order, *d_n <= n_max entries (device).
// Equal (cluster, term) are added in FP64 in the order given, then the new
// means follow as in launch_means_from_sums (u_max = n_max).
struct PartialArgs {
  int64_t n_max;
  const int64_t* d_n;
  const int32_t* cluster;
  const int32_t* term;
  const double* sum;
};
cudaError_t launch_update_from_partials(const UpdateArgs& a, const PartialArgs& p, cudaStream_t s);
// Every cluster id in [0, k) and term id in [0, d); a violation sets STS_BAD_ROWS.
cudaError_t launch_check_partials(int64_t n, const int32_t* cluster, const int32_t* term, int32_t k, int32_t d,
                                  unsigned* status, cudaStream_t s);

struct IvfBuildArgs {
  int64_t kt, dt, cap;
  int tbits;
  int32_t n_inst;
  const int32_t* inst_clu;
  const int64_t* mptr;   // [Kt+1]; mptr[Kt] = E
  const int32_t* mterm;
  const double* mval;
  const int32_t* mclu;
  int64_t* term_ptr;     // [Dt+1]
  uint16_t* cid16;
  int32_t* cid32;
  void* w;               // storage type
  int32_t storage;
  int32_t* toff;         // or null
  int32_t n_tiles_max, k_tile;
  int64_t* d_e;          // [1] receives E
  // dense head rows (null head_slot = off; single-instance contexts only)
  int32_t* head_slot;    // [Dt]
  void* wd;              // [head_max * kpad]
  int64_t kpad;
  int64_t head_max;      // rows available in wd
  int64_t head_min_nc;   // a list of at least this many clusters is stored densely
  float head_theta;      // ... or, with several instances, theta * K of the term's instance
  const int64_t* inst_toff;  // [n_inst+1] term offsets of the instances
  uint32_t* hflags;      // [Dt+1] scratch
  int64_t* d_heads;      // [1] receives the number of dense rows
  int64_t zero_rows;     // rows of wd cleared before filling (0: the rows in use)
  int64_t* d_heads_wanted;  // [1] receives the number of lists that qualified (may exceed head_max)
  void* wdT = nullptr;       // tensor-core head: transposed rows [kpad x ldt] (K-major B operand), or null
  int64_t ldt = 0;
  // scratch
  uint32_t* k32a;
  uint32_t* k32b;
  uint32_t* v32a;
  uint32_t* v32b;
  uint64_t* v64a;  // [cap] payloads of the rebuild sort
  uint64_t* v64b;
  void* temp;
  unsigned* status;
};
cudaError_t launch_build_ivf(const IvfBuildArgs& a, cudaStream_t s);
cudaError_t launch_build_toff(const IvfBuildArgs& a, cudaStream_t s);
cudaError_t launch_build_head(const IvfBuildArgs& a, cudaStream_t s);

// Means from rows: validate cluster-major rows, fill the row owner of every
// entry and (normalise != 0) divide each row by its FP64 L2 norm in place;
// a zero-norm row (when normalising) or a bad term sets STS_BAD_MEANS, a
// negative value sets *negative.
cudaError_t launch_normalise_rows(int64_t kt, const int64_t* mptr, double* mval, int32_t* mclu,
                                  int64_t dt, const int32_t* mterm, unsigned* status, int normalise,
                                  unsigned* negative, cudaStream_t s);
// Gather object rows d_ids[j] (global object ids) as mean rows (values promoted to FP64).
cudaError_t launch_gather_rows(int64_t kt, const int32_t* doc_ids, const int64_t* row_ptr,
                               const int32_t* term, const float* val32, int64_t* lens_then_ptr,
                               int32_t* mterm, double* mval, void* temp, cudaStream_t s, int phase);

// Object-side preparation: norms, storage copy, validation, and (term_rebase
// = term, non-null) global term ids written in place; with term_rebase null
// the rows are only read.
cudaError_t launch_prepare_objects(int64_t n_docs, int64_t nnz, int64_t dt_local_max, const int64_t* row_ptr,
                                   const int32_t* term, int32_t* term_rebase, const float* val32, void* val_store,
                                   int storage,
                                   float* nx, int32_t n_inst, const int64_t* inst_docs,
                                   const int64_t* inst_toff, const int32_t* inst_terms, int validate,
                                   unsigned* status, unsigned* negative, cudaStream_t s);

// Dense 16-bit head values of objects [i0, i0 + nb): x[(i - i0) * ldx + head_slot[t]] = val[h]
// for every head term t of object i, zeros elsewhere; chunk_nz (or null)
// [ceil(nb / 128) x ldx / 64] gets 1 for every (128-object block, 64-slot
// chunk) holding a value.
cudaError_t launch_build_xhead(int64_t i0, int64_t nb, const int64_t* row_ptr, const int32_t* term,
                               const void* val16, const int32_t* head_slot, void* x, int64_t ldx,
                               uint8_t* chunk_nz, cudaStream_t s);

// Tensor-core head product (tc_head.cu): d[i][c] = sum_s a[i][s] * b[c][s]
// for i < m, c < n, s < k; a, b 16-bit (both bf16 or both fp16), d 16-bit
// (bf16 or fp16), row-major with leading dimensions lda, ldb, ldd (elements,
// multiples of 8; pointers 16-byte aligned), FP32 accumulation, d rounded to
// its 16-bit type.
// n a multiple of 256, k a multiple of 64.  chunk_nz (or null): per
// 128-row block of a and 64-column chunk, 0 when that chunk of a is zero
// (skipped).  A bounded wait that runs out sets STS_TIMEOUT in *status.
struct TcHeadArgs {
  int64_t m;
  int32_t n, k;
  const void* a;
  int64_t lda;
  const void* b;
  int64_t ldb;
  void* d;
  int64_t ldd;
  bool bf16;      // a and b are bf16 (else fp16)
  bool out_bf16;  // d is bf16 (else fp16)
  const uint8_t* chunk_nz;
  unsigned* status;
  int num_sms;
};
cudaError_t launch_tc_head(const TcHeadArgs& h, cudaStream_t s);
// The objects' tuples in term-major order, ascending object inside each term
// (zeta): built once per object set by a stable sort of the CSR tuples by
// term; the update step groups it by cluster, IVFD walks it per term.
struct ZetaArgs {
  int64_t n_docs, nnz, dt;
  const int64_t* row_ptr;
  const int32_t* term;
  const float* val32;
  int64_t* zptr;    // [D+1]
  uint32_t* zterm;  // [nnz] term of each tuple
  uint64_t* zov;    // [nnz] object << 32 | FP32 value bits
  uint32_t* k32;    // [nnz] scratch keys
  uint64_t* v64;    // [nnz] scratch payloads
  void* temp;
  const int64_t* d_nnz;
  int tbits;        // bits of the (global) term ids
};
cudaError_t launch_build_zeta(const ZetaArgs& z, cudaStream_t s);

// ------------------------------------------------------------------ IVFD
// The comparison algorithm IVFD (Algorithm 4): objects also held as an
// inverted file zeta (term-major (object, value) lists in ascending object),
// assignment looping over the means (ivfd.cu).  FP32, one instance.
constexpr int IVFD_SUB = 512;  // objects per sub-range (one warp's accumulator)
struct IvfdArgs {
  int64_t n_docs, nnz, dt;
  int32_t k;
  const int64_t* row_ptr;
  const int32_t* term;
  const float* val32;
  const float* nx;
  // zeta, built once per object set: zptr [D+1], zov [nnz] (object << 32 |
  // value bits), zoff [D x (n_sub+1)] offset inside zeta_s of the first
  // object >= r * IVFD_SUB
  const int64_t* zptr;
  const uint64_t* zov;
  int32_t* zoff;
  int64_t n_sub;
  // the means, cluster-major FP64, and the inverted file's list bounds (for
  // the zero-similarity test)
  const int64_t* mptr;
  const int32_t* mterm;
  const double* mval;
  const int64_t* term_ptr;
  // per (chunk, object) top-2 of the chunk's means: [chunks x N]
  int32_t chunks;
  float* pbest;
  float* psecond;
  int32_t* pid;
  // outputs and counters, as for the IVF kernel
  int32_t* assign;
  float* best;
  float* gap;
  float* err;
  unsigned long long* entries;
  unsigned long long* n_zero_sim;
  int32_t rescore;
  unsigned int* n_flagged;
  int32_t* flag_obj;
  int32_t* flag_cnt;
  // near-ties: appended here (count *n_preflag) for an object-major IVF pass
  // that collects their candidates; null = re-scored against every cluster
  int32_t* preflag;
  unsigned int* n_preflag;
  int32_t nonneg;
  const unsigned* negative;
  const unsigned* means_negative;
};
int64_t ivfd_sub_ranges(int64_t n_docs);
// zoff from zeta (zptr, zobj must be built).
cudaError_t launch_build_ivfd_offsets(const IvfdArgs& a, cudaStream_t s);
cudaError_t launch_assign_ivfd(const IvfdArgs& a, cudaStream_t s);

// Transpose the dense head rows wd [rows x kpad] into wdT [kpad x ldt] (16-bit).
cudaError_t launch_transpose16(const void* wd, int64_t rows, int64_t kpad, void* wdT, int64_t ldt, cudaStream_t s);
cudaError_t launch_check_row_ptr(const int64_t* rp, int64_t n, int64_t nnz, unsigned* status, cudaStream_t s);

}  // namespace ivfk
