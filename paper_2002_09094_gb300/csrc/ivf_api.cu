// C ABI of libivfkm (include/ivf.h): context, device layout, autotuner,
// CUDA-graph iterations.  All arithmetic of the method runs in the kernels of
// assign.cu, update.cu, radix.cu and (FP16/BF16 tensor-core head) tc_head.cu;
// this file validates, allocates, copies and launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ivf.h"
#include "common.cuh"
#include "kernels.cuh"
#include "radix.cuh"

namespace ivfk {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace ivfk

using namespace ivfk;

namespace {

// Tile-major assignments launch once per accumulator tile, up to this many,
// and carry up to kTileCand re-score candidates per object between launches.
constexpr int kMaxTileLaunches = 128;
constexpr int kTileCand = 32;

// Counters the kernels update; one device block, mirrored into pinned host memory.
struct DevCounters {
  unsigned long long work;
  unsigned long long entries;
  unsigned long long n_rescored;
  unsigned long long work_cls[8];   // work counters of the per-class launches (batched contexts)
  unsigned long long zero_sim;      // objects that met no posting entry in the last assignment
  unsigned long long work_re;       // work counter of the object-major pass over near-ties
  unsigned long long entries_re;    // entries of that pass (already counted by the sweep)
  unsigned long long work_tile[kMaxTileLaunches];  // work counters of the tile-major launches
  unsigned int n_preflag;           // near-ties found by a tile-major sweep
  unsigned int n_flagged;
  unsigned int status;
  double objective;
  unsigned long long cnt[2];  // changed, zero-sim
  long long ivf_e;            // entries of the inverted file last built
  unsigned long long acc_entries;   // timing window sums
  unsigned long long acc_rescored;
  long long heads;                  // dense head rows of the inverted file last built
  unsigned int negative;            // some object value is negative (not an error)
  unsigned int means_negative[2];   // some value of means buffer 0 / 1 is negative
  long long heads_wanted;           // lists that qualified as dense rows in the last build
};

struct Shape {
  int tile_cap = 0;   // floats per warp
  int k_tile = 0;     // clusters per tile
  int tiled = 0;
  int warps = 0;
  int blocks = 0;
  int head_r = 0;     // registers per lane of the dense-head accumulator (0 = no dense head)
  int head_sub = 1;   // dense-head sub-tiles (32 * head_r clusters) per shared-memory tile
  bool tc = false;    // head part by a tensor-core GEMM (16-bit storage, one instance)
  float head_theta = 0.f;  // a list covering at least this fraction of K is stored densely
  // Tile-major schedule (tiled shapes): one launch per accumulator tile over
  // all objects, so the rows and list slices of one tile are what the SMs
  // share in L2 at a time; an object-major pass then collects the candidates
  // of the near-ties.
  bool tmajor = false;
};

// Dense head rows start with room for this much device memory and grow, when
// more lists qualify, up to kHeadMaxBytes.
constexpr int64_t kHeadBudgetBytes = int64_t(2) << 30;
constexpr int64_t kHeadMaxBytes = int64_t(24) << 30;

std::mutex g_tune_mu;
struct TuneChoice {
  Shape main;
  std::vector<Shape> cls;  // batched contexts: the classes below the last one
};
std::map<std::tuple<int64_t, int64_t, int64_t, int, int>, TuneChoice> g_tune_cache;

constexpr int kTileChoices[] = {1024, 2048, 4096, 8192, 16384, 32768};
constexpr size_t kSmemBudget = 227 * 1024;

}  // namespace

struct ivf_ctx {
  ivf_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  // sizes
  int64_t N = 0, nnz = 0, Dt = 0, Kt = 0;
  int32_t n_inst = 1;
  int32_t kmax = 0;
  int tbits = 1, kbits = 1;
  int tbits_local = 1;  // bits of the largest instance's own term ids (update-step sort keys)
  int64_t cap = 0;  // capacity of means / inverted-file arrays
  int64_t e_cur = 0;
  std::vector<int64_t> h_inst_docs, h_inst_toff;
  std::vector<int32_t> h_inst_clu, h_inst_terms;
  // allocations
  std::vector<void*> allocs;
  std::vector<int64_t> alloc_bytes;  // size of each entry of allocs
  int64_t bytes = 0;
  // objects
  int64_t* row_ptr = nullptr;
  int32_t* term = nullptr;
  float* val32 = nullptr;
  void* val_store = nullptr;
  float* nx = nullptr;
  // staging copy of the objects for ivf_load_objects: filled on copy_stream
  // (ev_staged), moved into place on the context stream by commit_objects
  // (ev_staging_free once those device copies ran)
  bool staging_ready = false;
  bool objects_pending = false;
  int64_t* st_row_ptr = nullptr;
  int32_t* st_term = nullptr;
  float* st_val32 = nullptr;
  unsigned* d_load_status = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_src = nullptr, ev_staged = nullptr, ev_staging_free = nullptr;
  int64_t* inst_docs = nullptr;
  int32_t* inst_clu = nullptr;
  int64_t* inst_toff = nullptr;
  int32_t* inst_terms = nullptr;
  // means, double buffered
  int64_t* mptr[2] = {nullptr, nullptr};
  int32_t* mterm[2] = {nullptr, nullptr};
  double* mval[2] = {nullptr, nullptr};
  int32_t* mclu[2] = {nullptr, nullptr};
  int mcur = 0;
  // inverted file
  int64_t* term_ptr = nullptr;
  uint16_t* cid16 = nullptr;
  int32_t* cid32 = nullptr;
  void* w = nullptr;
  int32_t* toff = nullptr;
  int64_t toff_len = 0;
  int64_t* d_e = nullptr;  // points into dc
  // dense head rows
  int32_t* head_slot = nullptr;
  uint32_t* hflags = nullptr;
  void* wd = nullptr;
  int64_t kpad = 0;
  int64_t head_max = 0;
  // assignment
  int32_t* assign[2] = {nullptr, nullptr};
  int alatest = -1;  // buffer holding the latest assignment, -1 = none
  bool has_prev_for_next = false;
  float* best = nullptr;
  float* gap = nullptr;
  float* errb = nullptr;  // per object: bound on |best - rho_FP64|
  int32_t* preflag = nullptr;  // near-ties of a tile-major sweep
  int64_t run_cap = 0;         // entries of flags / starts (+1) and ukey / usum
  // member sums gathered from shards (ivf_update_from_partials)
  int32_t* part_cluster = nullptr;
  int32_t* part_term = nullptr;
  double* part_sum = nullptr;
  int64_t part_cap = 0, part_n = 0;
  int64_t* d_part_n = nullptr;
  // candidate carry of tile-major sweeps: [N x kTileCand] ids and values, [N] counts
  int32_t* tcand = nullptr;
  float* tcandv = nullptr;
  int32_t* tcand_n = nullptr;
  // zeta: the objects' tuples in term-major order (term, and object << 32 |
  // value bits, ascending object inside each term), rebuilt with the objects;
  // the update step sorts it by cluster, IVFD reads it as the objects'
  // inverted file
  int64_t* zptr = nullptr;
  uint32_t* zterm = nullptr;
  uint64_t* zov = nullptr;
  // IVFD (IVF_FLAG_IVFD): per-(term, sub-range) offsets into zeta, built once
  // per object set, and the per-(mean chunk, object) top-2
  bool ivfd_built = false;
  int32_t* zoff = nullptr;
  int64_t z_sub = 0;
  int32_t z_chunks = 0;
  float* z_pbest = nullptr;
  float* z_psecond = nullptr;
  int32_t* z_pid = nullptr;
  int32_t* flag_obj = nullptr;
  int32_t* flag_cnt = nullptr;
  int32_t* flag_cand = nullptr;
  DevCounters* dc = nullptr;
  DevCounters* hc = nullptr;  // pinned
  int red_blocks = 0;
  double* part_obj = nullptr;
  unsigned long long* part_cnt = nullptr;
  long long* inst_changed = nullptr;
  // members
  int64_t* cl_ptr = nullptr;
  int32_t* members = nullptr;
  double* sum_norm = nullptr;
  double* rnorm = nullptr;
  bool members_valid = false;
  // update scratch
  uint64_t* k64a = nullptr;
  uint64_t* k64b = nullptr;
  uint32_t* v32a = nullptr;
  uint32_t* v32b = nullptr;
  uint32_t* flags = nullptr;
  uint32_t* starts = nullptr;
  uint64_t* ukey = nullptr;
  double* usum = nullptr;
  int64_t* uptr = nullptr;
  int64_t* newlen = nullptr;
  int32_t* zrun = nullptr;
  int64_t* d_nnz = nullptr;
  int64_t* d_n = nullptr;
  int64_t* d_u = nullptr;
  void* temp = nullptr;
  int64_t scratch_len = 0;
  // launch shape (of the class holding the largest K in a batched context)
  Shape shape;
  // Batched contexts: instances grouped by K (<= 128, <= 256, <= 512, <= 1,024,
  // <= 1,536, <= 2,048, larger), one
  // assignment launch per class, each with its own kernel; the last class
  // holds the largest K and uses `shape` (the only one that may be tiled).
  struct ClassPlan {
    int32_t kmax = 0;
    int64_t n_objs = 0;
    std::vector<int32_t> insts;
    int32_t* d_inst = nullptr;
    int64_t* d_prefix = nullptr;
    Shape shape;
  };
  std::vector<ClassPlan> cls;
  bool use_classes = false;
  // tensor-core head: objects in batches of tc_batch; per batch the dense
  // head values xh [tc_batch x head_max] with their nonzero-chunk flags, and
  // the product rho_h [tc_batch x kpad] (16-bit, the storage type); the dense
  // rows transposed, wdT [kpad x head_max] (the K-major B operand)
  void* xh = nullptr;
  void* rho_h = nullptr;
  void* wdT = nullptr;
  uint8_t* chunk_nz = nullptr;
  int64_t tc_batch = 0;
  int64_t tc_alloc_rows = 0, tc_alloc_kpad = 0, tc_alloc_batch = 0;
  bool tuned = false;
  bool tuned_on_updated_means = false;  // the choice was made on means from an update step
  int64_t e_tuned = 0;   // inverted-file entries when the choice was made
  int32_t tunings = 0;   // choices made so far (bounded)
  // state
  bool means_set = false;
  int64_t cand_slots = 0;      // flagged objects with room for a candidate list
  int32_t iteration = 0;
  // graphs keyed by (mcur, alatest)
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  long long graph_kernels[2][2] = {{0, 0}, {0, 0}};
  bool own_stream = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};  // assignment start / end
  // timing window: event pool and per-call records
  bool timing = false;
  std::vector<cudaEvent_t> tev;
  size_t tev_used = 0;
  struct TimedCall {
    int kind;  // 0 assign (3 events), 1 update (2 events)
    size_t e0;
  };
  std::vector<TimedCall> tcalls;
};

namespace {

ivf_status fail(ivf_ctx* c, ivf_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

ivf_status fail_cuda(ivf_ctx* c, const char* what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return fail(c, IVF_E_CUDA, buf);
}

#define CK(c, expr)                                        \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return fail_cuda((c), #expr, e_); \
  } while (0)

#define ST(expr)                     \
  do {                               \
    ivf_status s_ = (expr);          \
    if (s_ != IVF_OK) return s_;     \
  } while (0)

template <typename T>
ivf_status dalloc(ivf_ctx* c, T** p, int64_t count) {
  const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof(buf), "cudaMalloc of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    return fail(c, IVF_E_OOM, buf);
  }
  c->allocs.push_back(q);
  c->alloc_bytes.push_back((int64_t)bytes);
  c->bytes += (int64_t)bytes;
  *p = static_cast<T*>(q);
  return IVF_OK;
}

void dfree(ivf_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) {
    const size_t k = (size_t)(it - c->allocs.begin());
    c->bytes -= c->alloc_bytes[k];
    c->alloc_bytes.erase(c->alloc_bytes.begin() + (std::ptrdiff_t)k);
    c->allocs.erase(it);
    cudaFree(p);
  }
}

size_t storage_bytes(int st) { return st == IVF_F32 ? 4 : 2; }

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

void drop_graphs(ivf_ctx* c) {
  for (auto& row : c->graph)
    for (auto& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

// Means / inverted-file arrays sized for `cap` entries.
ivf_status alloc_means(ivf_ctx* c, int64_t cap) {
  for (int b = 0; b < 2; ++b) {
    dfree(c, c->mterm[b]);
    dfree(c, c->mval[b]);
    dfree(c, c->mclu[b]);
    c->mterm[b] = nullptr;
    c->mval[b] = nullptr;
    c->mclu[b] = nullptr;
  }
  dfree(c, c->cid16);
  dfree(c, c->cid32);
  dfree(c, c->w);
  c->cid16 = nullptr;
  c->cid32 = nullptr;
  c->w = nullptr;
  for (int b = 0; b < 2; ++b) {
    ST(dalloc(c, &c->mterm[b], cap));
    ST(dalloc(c, &c->mval[b], cap));
    ST(dalloc(c, &c->mclu[b], cap));
  }
  ST(dalloc(c, &c->cid16, cap + 8));
  ST(dalloc(c, &c->cid32, cap));
  char* wp = nullptr;
  ST(dalloc(c, &wp, (cap + 8) * (int64_t)storage_bytes(c->cfg.storage)));
  c->w = wp;
  c->cap = cap;
  drop_graphs(c);
  return IVF_OK;
}

ivf_status alloc_scratch(ivf_ctx* c, int64_t len) {
  void* olds[] = {c->k64a, c->k64b, c->v32a, c->v32b, c->temp};
  for (void* p : olds) dfree(c, p);
  ST(dalloc(c, &c->k64a, len));
  ST(dalloc(c, &c->k64b, len));
  ST(dalloc(c, &c->v32a, len));
  ST(dalloc(c, &c->v32b, len));
  size_t tb = std::max({radix_temp_bytes(len), scan_temp_bytes(len + 1), scan_temp_bytes(c->Kt + 1),
                        scan_temp_bytes(c->Dt + 1)});
  char* t = nullptr;
  ST(dalloc(c, &t, (int64_t)tb));
  c->temp = t;
  c->scratch_len = len;
  drop_graphs(c);
  return IVF_OK;
}

ivf_status check_status(ivf_ctx* c) {
  unsigned st = 0;
  CK(c, cudaMemcpyAsync(&st, &c->dc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (st) {
    CK(c, cudaMemsetAsync(&c->dc->status, 0, sizeof(unsigned), c->stream));
    if (st & STS_CAPACITY) return fail(c, IVF_E_OOM, "new means exceed the inverted-file capacity");
    if (st & STS_BAD_MEANS) return fail(c, IVF_E_INVALID, "a mean row has zero norm, bad or unsorted terms");
    if (st & STS_BAD_ROWS) return fail(c, IVF_E_INVALID, "object rows failed validation");
    if (st & STS_TIMEOUT) return fail(c, IVF_E_TIMEOUT, "a bounded device wait ran out (tensor-core head)");
    return fail(c, IVF_E_INVALID, "device status error");
  }
  return IVF_OK;
}

// --------------------------------------------------------------- create

ivf_status enqueue_build_zeta(ivf_ctx* c);

ivf_status create_common(const ivf_config* cfg, int32_t n_inst, const std::vector<int64_t>& inst_docs,
                         const std::vector<int32_t>& inst_terms, const std::vector<int32_t>& inst_k,
                         const int64_t* row_ptr, const int32_t* term, const float* val, void* stream,
                         ivf_ctx** out) {
  ivf_ctx* c = new ivf_ctx();
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(stream);
  c->n_inst = n_inst;
  auto bail = [&](ivf_status s) {
    if (s != IVF_OK && c->err.size()) fprintf(stderr, "libivfkm: %s\n", c->err.c_str());
    ivf_destroy(c);
    return s;
  };
  if (!c->stream) {
    // The legacy default stream cannot be captured into a graph: work goes to
    // a private blocking stream, which the legacy stream orders implicitly.
    cudaError_t es = cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault);
    if (es != cudaSuccess) return bail(fail_cuda(c, "cudaStreamCreate", es));
    c->own_stream = true;
  }
  {
    cudaError_t er = radix_prepare();
    if (er != cudaSuccess) return bail(fail_cuda(c, "radix_prepare", er));
  }
  // instance tables
  c->h_inst_docs = inst_docs;
  c->h_inst_terms = inst_terms;
  c->h_inst_clu.assign(n_inst + 1, 0);
  c->h_inst_toff.assign(n_inst + 1, 0);
  for (int b = 0; b < n_inst; ++b) {
    c->h_inst_clu[b + 1] = c->h_inst_clu[b] + inst_k[b];
    c->h_inst_toff[b + 1] = c->h_inst_toff[b] + inst_terms[b];
    c->kmax = std::max(c->kmax, inst_k[b]);
  }
  c->N = inst_docs[n_inst];
  c->Kt = c->h_inst_clu[n_inst];
  c->Dt = c->h_inst_toff[n_inst];
  c->tbits = bits_for(c->Dt);
  c->kbits = bits_for(c->Kt);
  c->tbits_local = bits_for(*std::max_element(inst_terms.begin(), inst_terms.end()));
  if (c->tbits + c->kbits > 64) return bail(fail(c, IVF_E_UNSUPPORTED, "cluster and term ids need more than 64 bits"));
  if (c->N >= (int64_t(1) << 31) || c->Kt >= (int64_t(1) << 31) || c->Dt >= (int64_t(1) << 31))
    return bail(fail(c, IVF_E_UNSUPPORTED, "N, K and D must be below 2^31"));

  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(fail_cuda(c, "cudaGetDevice", e));
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(fail_cuda(c, "cudaDeviceGetAttribute", e));

  // row_ptr checked on the host
  std::vector<int64_t> hrp(c->N + 1);
  e = cudaMemcpy(hrp.data(), row_ptr, sizeof(int64_t) * (c->N + 1), cudaMemcpyDefault);
  if (e != cudaSuccess) return bail(fail_cuda(c, "copy row_ptr", e));
  if (hrp[0] != 0) return bail(fail(c, IVF_E_INVALID, "row_ptr[0] must be 0"));
  for (int64_t i = 0; i < c->N; ++i)
    if (hrp[i + 1] < hrp[i]) return bail(fail(c, IVF_E_INVALID, "row_ptr must be non-decreasing"));
  c->nnz = hrp[c->N];
  if (cfg->nnz >= 0 && n_inst == 1 && cfg->nnz != c->nnz)
    return bail(fail(c, IVF_E_INVALID, "row_ptr[N] differs from cfg->nnz"));
  if (c->nnz >= (int64_t(1) << 32) - 2) return bail(fail(c, IVF_E_UNSUPPORTED, "nnz must be below 2^32"));
  for (int b = 0; b < n_inst; ++b)
    if (hrp[inst_docs[b + 1]] - hrp[inst_docs[b]] > (int64_t)inst_terms[b] * (inst_docs[b + 1] - inst_docs[b]))
      return bail(fail(c, IVF_E_INVALID, "more tuples than terms allow"));

  const int64_t N = c->N, nnz = c->nnz;
  ivf_status s;
#define AL(p, n)                    \
  if ((s = dalloc(c, &(p), (n))) != IVF_OK) return bail(s);
  AL(c->row_ptr, N + 1);
  AL(c->term, nnz);
  AL(c->val32, nnz);
  if (cfg->storage != IVF_F32) {
    char* vs = nullptr;
    AL(vs, nnz * 2 + 16);
    c->val_store = vs;
  } else {
    c->val_store = c->val32;
  }
  AL(c->nx, N);
  AL(c->inst_docs, n_inst + 1);
  AL(c->inst_clu, n_inst + 1);
  AL(c->inst_toff, n_inst + 1);
  AL(c->inst_terms, n_inst);
  for (int b = 0; b < 2; ++b) AL(c->mptr[b], c->Kt + 1);
  AL(c->term_ptr, c->Dt + 1);
  for (int b = 0; b < 2; ++b) AL(c->assign[b], N);
  AL(c->best, N);
  AL(c->gap, N);
  AL(c->errb, N);
  AL(c->preflag, N);
  AL(c->flag_obj, N);
  AL(c->flag_cnt, N);
  c->cand_slots = std::min<int64_t>(N, int64_t(1) << 20);
  // batched: classes of instances by K (see ClassPlan); autotuned contexts only
  if (n_inst > 1 && cfg->k_tile == 0 && cfg->warps_per_block == 0) {
    // classes by K: each gets its own kernel (tiny K favours the sparse
    // kernel, larger K the dense-head register tiles; above 1,024 clusters
    // the best split of the 2,048-cluster tile -- 4 x 512 or 2 x 1,024 --
    // changes with K)
    constexpr int kClasses = 7;
    const int32_t bounds[kClasses] = {128, 256, 512, 1024, 1536, 2048, INT32_MAX};
    for (int32_t lo = 0, q = 0; q < kClasses; lo = bounds[q], ++q) {
      ivf_ctx::ClassPlan p;
      std::vector<int64_t> prefix(1, 0);
      for (int32_t b = 0; b < n_inst; ++b)
        if (inst_k[b] > lo && inst_k[b] <= bounds[q]) {
          p.insts.push_back(b);
          prefix.push_back(prefix.back() + (inst_docs[b + 1] - inst_docs[b]));
          p.kmax = std::max(p.kmax, inst_k[b]);
        }
      if (p.insts.empty()) continue;
      p.n_objs = prefix.back();
      AL(p.d_inst, (int64_t)p.insts.size());
      AL(p.d_prefix, (int64_t)prefix.size());
      e = cudaMemcpy(p.d_inst, p.insts.data(), sizeof(int32_t) * p.insts.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(p.d_prefix, prefix.data(), sizeof(int64_t) * prefix.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return bail(fail_cuda(c, "cudaMemcpy", e));
      c->cls.push_back(std::move(p));
    }
    c->use_classes = c->cls.size() > 1;
    if (!c->use_classes) c->cls.clear();
  }
  AL(c->flag_cand, c->cand_slots * (int64_t)CAND_MAX);
  AL(c->dc, 1);
  c->d_e = reinterpret_cast<int64_t*>(&c->dc->ivf_e);
  c->red_blocks = (int)std::min<int64_t>(ceil_div(N, 256), 4 * (int64_t)c->num_sms);
  if (c->red_blocks < 1) c->red_blocks = 1;
  AL(c->part_obj, c->red_blocks);
  AL(c->part_cnt, 2 * (int64_t)c->red_blocks);
  AL(c->inst_changed, n_inst);
  AL(c->cl_ptr, c->Kt + 1);
  AL(c->members, N);
  AL(c->sum_norm, c->Kt);
  AL(c->rnorm, c->Kt);
  AL(c->flags, nnz + 1);
  AL(c->starts, nnz + 1);
  AL(c->ukey, nnz);
  AL(c->usum, nnz);
  c->run_cap = nnz;
  AL(c->d_part_n, 1);
  AL(c->uptr, c->Kt + 1);
  AL(c->newlen, c->Kt + 1);
  AL(c->zrun, c->Kt);
  AL(c->d_nnz, 1);
  AL(c->d_n, 1);
  AL(c->d_u, 1);
  AL(c->zptr, c->Dt + 1);
  AL(c->zterm, std::max<int64_t>(1, nnz));
  AL(c->zov, std::max<int64_t>(1, nnz));
#undef AL
  e = cudaMallocHost(&c->hc, sizeof(DevCounters));
  if (e != cudaSuccess) return bail(fail_cuda(c, "cudaMallocHost", e));
  for (auto& ev : c->ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return bail(fail_cuda(c, "cudaEventCreate", e));
  }
  // The means rarely need more entries than half the tuples; very large
  // problems start there and grow on demand (grow_means), smaller ones get room.
  const int64_t cap0 = cfg->means_capacity > 0 ? (int64_t)cfg->means_capacity
                       : nnz > (int64_t(400) << 20) ? nnz / 2 + 4096
                                                     : nnz + nnz / 4 + 4096;
  if ((s = alloc_means(c, cap0)) != IVF_OK) return bail(s);
  if ((s = alloc_scratch(c, std::max<int64_t>({nnz, c->cap, N + 1}))) != IVF_OK) return bail(s);

  cudaStream_t st = c->stream;
#define CKB(expr)                                   \
  do {                                              \
    cudaError_t e2 = (expr);                        \
    if (e2 != cudaSuccess) return bail(fail_cuda(c, #expr, e2)); \
  } while (0)
  CKB(cudaMemsetAsync(c->dc, 0, sizeof(DevCounters), st));
  CKB(cudaMemcpyAsync(c->row_ptr, hrp.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(c->term, term, sizeof(int32_t) * nnz, cudaMemcpyDefault, st));
  CKB(cudaMemcpyAsync(c->val32, val, sizeof(float) * nnz, cudaMemcpyDefault, st));
  CKB(cudaMemcpyAsync(c->inst_docs, c->h_inst_docs.data(), sizeof(int64_t) * (n_inst + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(c->inst_clu, c->h_inst_clu.data(), sizeof(int32_t) * (n_inst + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(c->inst_toff, c->h_inst_toff.data(), sizeof(int64_t) * (n_inst + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(c->inst_terms, c->h_inst_terms.data(), sizeof(int32_t) * n_inst, cudaMemcpyHostToDevice, st));
  const int64_t dn[2] = {nnz, N};
  CKB(cudaMemcpyAsync(c->d_nnz, &dn[0], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(c->d_n, &dn[1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CKB(launch_prepare_objects(N, nnz, 0, c->row_ptr, c->term, c->term, c->val32,
                             cfg->storage == IVF_F32 ? nullptr : c->val_store, cfg->storage, c->nx, n_inst,
                             c->inst_docs, c->inst_toff, c->inst_terms, (cfg->flags & IVF_FLAG_VALIDATE) ? 1 : 0,
                             &c->dc->status, &c->dc->negative, st));
#undef CKB
  if ((s = check_status(c)) != IVF_OK) return bail(s);
  if ((s = enqueue_build_zeta(c)) != IVF_OK) return bail(s);
  *out = c;
  return IVF_OK;
}

ivf_status validate_cfg(const ivf_config* cfg) {
  if (!cfg) return IVF_E_INVALID;
  if (cfg->storage < IVF_F32 || cfg->storage > IVF_BF16) return IVF_E_INVALID;
  if (cfg->empty_policy != 0 && cfg->empty_policy != 1) return IVF_E_INVALID;
  if (cfg->rescore != 0 && cfg->rescore != 1) return IVF_E_INVALID;
  if (cfg->warps_per_block < 0 || cfg->warps_per_block > 32) return IVF_E_INVALID;
  if (cfg->means_capacity < 0) return IVF_E_INVALID;
  if (cfg->dense_head_bytes < 0) return IVF_E_INVALID;
  if (cfg->k_tile < 0) return IVF_E_INVALID;
  if ((cfg->flags & IVF_FLAG_IVFD) && cfg->storage != IVF_F32) return IVF_E_UNSUPPORTED;
  return IVF_OK;
}

// ---------------------------------------------------------- inverted file

IvfBuildArgs ivf_args(ivf_ctx* c, int mb) {
  IvfBuildArgs a{};
  a.kt = c->Kt;
  a.dt = c->Dt;
  a.cap = c->cap;
  a.tbits = c->tbits;
  a.n_inst = c->n_inst;
  a.inst_clu = c->inst_clu;
  a.mptr = c->mptr[mb];
  a.mterm = c->mterm[mb];
  a.mval = c->mval[mb];
  a.mclu = c->mclu[mb];
  a.term_ptr = c->term_ptr;
  a.cid16 = c->cid16;
  a.cid32 = c->cid32;
  a.w = c->w;
  a.storage = c->cfg.storage;
  a.toff = c->shape.tiled ? c->toff : nullptr;
  a.k_tile = c->shape.k_tile;
  a.n_tiles_max = c->shape.tiled ? (int32_t)ceil_div(c->kmax, c->shape.k_tile) : 0;
  a.d_e = c->d_e;
  a.k32a = reinterpret_cast<uint32_t*>(c->k64a);
  a.k32b = reinterpret_cast<uint32_t*>(c->k64b);
  a.v32a = c->v32a;
  a.v32b = c->v32b;
  a.v64a = c->k64a;
  a.v64b = c->k64b;
  a.temp = c->temp;
  a.status = &c->dc->status;
  if (c->shape.head_r > 0 && c->head_slot) {
    a.head_slot = c->head_slot;
    a.wd = c->wd;
    a.kpad = c->kpad;
    a.head_max = c->head_max;
    a.head_min_nc = std::max<int64_t>(1, (int64_t)std::ceil((double)c->shape.head_theta * c->kmax));
    a.head_theta = c->shape.head_theta;
    a.inst_toff = c->inst_toff;
    a.hflags = c->hflags;
    a.d_heads = reinterpret_cast<int64_t*>(&c->dc->heads);
    a.zero_rows = c->shape.tc ? c->head_max : 0;  // the GEMM reads every row
    a.d_heads_wanted = reinterpret_cast<int64_t*>(&c->dc->heads_wanted);
    if (c->shape.tc && c->wdT) {
      a.wdT = c->wdT;
      a.ldt = c->head_max;
    }
  }
  return a;
}

// Buffers of the dense head rows for tiles of 32 * head_r clusters.
ivf_status alloc_head(ivf_ctx* c, int head_r) {
  // batched contexts: rows padded to 1,024 clusters, so every class may use
  // any register tile with the rows built for the largest class
  const int64_t tile = 32 * (int64_t)(c->n_inst > 1 ? HEAD_R_LARGE : head_r);
  const int64_t kpad = ceil_div(c->kmax, tile) * tile;
  if (c->head_slot && c->kpad == kpad) return IVF_OK;
  dfree(c, c->head_slot);
  dfree(c, c->hflags);
  dfree(c, c->wd);
  c->head_slot = nullptr;
  c->hflags = nullptr;
  c->wd = nullptr;
  const int64_t vb = (int64_t)storage_bytes(c->cfg.storage);
  const int64_t budget = c->cfg.dense_head_bytes > 0 ? c->cfg.dense_head_bytes : kHeadBudgetBytes;
  c->head_max = std::max<int64_t>(1, std::min<int64_t>(c->Dt, budget / (kpad * vb)));
  c->kpad = kpad;
  ST(dalloc(c, &c->head_slot, c->Dt));
  ST(dalloc(c, &c->hflags, c->Dt + 1));
  char* p = nullptr;
  ST(dalloc(c, &p, c->head_max * kpad * vb));
  c->wd = p;
  drop_graphs(c);
  return IVF_OK;
}

// When more lists qualified as dense rows in the last build (wanted) than
// the rows hold, grow the rows (up to kHeadMaxBytes) and rebuild them from
// the current means; the lists that did not fit were read sparsely, which is
// exact but slower.  Synchronises only when it grows.
ivf_status grow_head_if_needed(ivf_ctx* c, long long wanted) {
  // (the tensor-core head keeps its row count: the GEMM's depth is fixed)
  if (c->shape.head_r <= 0 || c->shape.tc || !c->head_slot || wanted <= c->head_max) return IVF_OK;
  const int64_t vb = (int64_t)storage_bytes(c->cfg.storage);
  const int64_t cap_rows = std::max<int64_t>(1, kHeadMaxBytes / (c->kpad * vb));
  const int64_t rows = std::min<int64_t>({c->Dt, cap_rows, (int64_t)wanted + wanted / 4 + 64});
  if (rows <= c->head_max) return IVF_OK;
  CK(c, cudaStreamSynchronize(c->stream));
  dfree(c, c->wd);
  c->wd = nullptr;
  char* p = nullptr;
  ST(dalloc(c, &p, rows * c->kpad * vb));
  c->wd = p;
  c->head_max = rows;
  drop_graphs(c);
  CK(c, launch_build_head(ivf_args(c, c->mcur), c->stream));
  return IVF_OK;
}

// Staging buffers, copy stream and events of ivf_load_objects (on first use).
ivf_status ensure_staging(ivf_ctx* c) {
  if (c->staging_ready) return IVF_OK;
  ST(dalloc(c, &c->st_row_ptr, c->N + 1));
  ST(dalloc(c, &c->st_term, c->nnz));
  ST(dalloc(c, &c->st_val32, c->nnz));
  ST(dalloc(c, &c->d_load_status, 1));
  if (!c->copy_stream) CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&c->ev_src, &c->ev_staged, &c->ev_staging_free})
    if (!*e) CK(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  c->staging_ready = true;
  return IVF_OK;
}

bool device_resident(const void* p) {
  cudaPointerAttributes at{};
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Objects loaded by ivf_load_objects take effect here, in stream order: the
// context stream waits for the staging copy, copies it into place (device to
// device) and prepares it as at create time.  Called by the calls that start
// from the objects (assignment, iterate, initial means from documents); the
// update step keeps working on the objects its assignment ran on.
IvfdArgs ivfd_args(ivf_ctx* c, int target, int rescore) {
  IvfdArgs a{};
  a.n_docs = c->N;
  a.nnz = c->nnz;
  a.dt = c->Dt;
  a.k = (int32_t)c->Kt;
  a.row_ptr = c->row_ptr;
  a.term = c->term;
  a.val32 = c->val32;
  a.nx = c->nx;
  a.zptr = c->zptr;
  a.zov = c->zov;
  a.zoff = c->zoff;
  a.n_sub = c->z_sub;
  a.mptr = c->mptr[c->mcur];
  a.mterm = c->mterm[c->mcur];
  a.mval = c->mval[c->mcur];
  a.term_ptr = c->term_ptr;
  a.chunks = c->z_chunks;
  a.pbest = c->z_pbest;
  a.psecond = c->z_psecond;
  a.pid = c->z_pid;
  a.assign = c->assign[target];
  a.best = c->best;
  a.gap = c->gap;
  a.err = c->errb;
  a.entries = &c->dc->entries;
  a.n_zero_sim = &c->dc->zero_sim;
  a.rescore = rescore;
  a.n_flagged = &c->dc->n_flagged;
  a.flag_obj = c->flag_obj;
  a.flag_cnt = c->flag_cnt;
  a.preflag = c->preflag;
  a.n_preflag = &c->dc->n_preflag;
  a.nonneg = 1;
  a.negative = &c->dc->negative;
  a.means_negative = &c->dc->means_negative[c->mcur];
  return a;
}

ivf_status commit_objects(ivf_ctx* c) {
  if (!c->objects_pending) return IVF_OK;
  c->objects_pending = false;
  cudaStream_t s = c->stream;
  CK(c, cudaStreamWaitEvent(s, c->ev_staged, 0));
  CK(c, cudaMemcpyAsync(c->row_ptr, c->st_row_ptr, sizeof(int64_t) * (c->N + 1), cudaMemcpyDeviceToDevice, s));
  CK(c, cudaMemcpyAsync(c->term, c->st_term, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToDevice, s));
  CK(c, cudaMemcpyAsync(c->val32, c->st_val32, sizeof(float) * c->nnz, cudaMemcpyDeviceToDevice, s));
  CK(c, cudaEventRecord(c->ev_staging_free, s));
  CK(c, cudaMemsetAsync(&c->dc->negative, 0, sizeof(unsigned), s));
  CK(c, launch_prepare_objects(c->N, c->nnz, 0, c->row_ptr, c->term, c->term, c->val32,
                               c->cfg.storage == IVF_F32 ? nullptr : c->val_store, c->cfg.storage, c->nx, c->n_inst,
                               c->inst_docs, c->inst_toff, c->inst_terms, (c->cfg.flags & IVF_FLAG_VALIDATE) ? 1 : 0,
                               &c->dc->status, &c->dc->negative, s));
  if (c->cfg.flags & IVF_FLAG_VALIDATE) ST(check_status(c));
  ST(enqueue_build_zeta(c));
  c->members_valid = false;
  c->ivfd_built = false;
  return IVF_OK;
}

// IVFD: zeta and its offsets for the current objects (allocates on first use;
// called before any stream capture).
ivf_status ensure_ivfd(ivf_ctx* c) {
  if (c->ivfd_built) return IVF_OK;
  if (!c->zoff) {
    c->z_sub = ivfd_sub_ranges(c->N);
    c->z_chunks = (int32_t)std::max<int64_t>(1, std::min<int64_t>(c->Kt, ceil_div(64 * (int64_t)c->num_sms, c->z_sub)));
    ST(dalloc(c, &c->zoff, c->Dt * (c->z_sub + 1)));
    ST(dalloc(c, &c->z_pbest, c->z_chunks * c->N));
    ST(dalloc(c, &c->z_psecond, c->z_chunks * c->N));
    ST(dalloc(c, &c->z_pid, c->z_chunks * c->N));
  }
  IvfdArgs a = ivfd_args(c, 0, 0);
  CK(c, launch_build_ivfd_offsets(a, c->stream));
  c->ivfd_built = true;
  return IVF_OK;
}

// zeta of the current objects (stream-ordered; after every object load).
ivf_status enqueue_build_zeta(ivf_ctx* c) {
  ZetaArgs z{};
  z.n_docs = c->N;
  z.nnz = c->nnz;
  z.dt = c->Dt;
  z.row_ptr = c->row_ptr;
  z.term = c->term;
  z.val32 = c->val32;
  z.zptr = c->zptr;
  z.zterm = c->zterm;
  z.zov = c->zov;
  z.k32 = c->v32a;
  z.v64 = c->k64a;
  z.temp = c->temp;
  z.d_nnz = c->d_nnz;
  z.tbits = c->tbits;
  CK(c, launch_build_zeta(z, c->stream));
  return IVF_OK;
}

// Stream-ordered: rebuild the inverted file from means buffer mb.
ivf_status enqueue_build_ivf(ivf_ctx* c, int mb) {
  CK(c, launch_build_ivf(ivf_args(c, mb), c->stream));
  return IVF_OK;
}

// ------------------------------------------------------------ autotune

AssignArgs assign_args(ivf_ctx* c, const Shape& sh, int target, int rescore) {
  AssignArgs a{};
  a.n_docs = c->N;
  a.row_ptr = c->row_ptr;
  a.term = c->term;
  a.val = c->val_store;
  a.nx = c->nx;
  a.n_inst = c->n_inst;
  a.inst_docs = c->inst_docs;
  a.inst_clu = c->inst_clu;
  a.term_ptr = c->term_ptr;
  a.cid = c->cid16;
  a.w = c->w;
  a.toff = sh.tiled ? c->toff : nullptr;
  a.n_tiles_max = sh.tiled ? (int32_t)ceil_div(c->kmax, sh.k_tile) : 0;
  a.k_tile = sh.k_tile;
  a.tiled = sh.tiled;
  a.tile_cap = sh.tile_cap;
  a.storage = c->cfg.storage;
  a.rescore = rescore;
  a.assign = c->assign[target];
  a.best = c->best;
  a.gap = c->gap;
  a.err = c->errb;
  a.work = &c->dc->work;
  a.entries = &c->dc->entries;
  a.n_zero_sim = &c->dc->zero_sim;
  a.n_flagged = &c->dc->n_flagged;
  a.flag_obj = c->flag_obj;
  a.flag_cnt = c->flag_cnt;
  a.flag_cand = c->flag_cand;
  a.cand_slots = c->cand_slots;
  // the kernel reads the sign flags of the objects and of the means buffer
  // the inverted file was built from, so no host copy of them is needed
  a.nonneg = 1;
  a.negative = &c->dc->negative;
  a.means_negative = &c->dc->means_negative[c->mcur];
  if (sh.head_r > 0) {
    a.head_slot = c->head_slot;
    a.wd = c->wd;
    a.kpad = c->kpad;
    a.head_sub = sh.head_sub;
  }
  return a;
}

// head_r > 0 selects the dense-head kernel, whose shared-memory tile is
// head_sub sub-tiles of 32 * head_r clusters.
bool shape_for(ivf_ctx* c, int32_t kmax, int k_tile, int warps_req, Shape* out, int head_r = 0, float theta = 0.f,
               int head_sub = 1, bool tc = false) {
  Shape sh;
  if (head_r > 0) {
    if (head_sub < 1 || !is_pow2(head_sub)) return false;
    k_tile = 32 * head_r * head_sub;
  }
  if (k_tile <= 0 || k_tile >= kmax) {
    if (kmax > 65536) return false;
    if (head_r > 0 && head_sub > 1 && 32 * head_r * (head_sub / 2) >= kmax) return false;  // no gain
    sh.tiled = 0;
    sh.k_tile = kmax;
    sh.tile_cap = (kmax + 3) & ~3;
  } else {
    if (!is_pow2(k_tile) || k_tile < (head_r > 0 ? 256 : 512) || k_tile > 65536) return false;
    sh.tiled = 1;
    sh.k_tile = k_tile;
    sh.tile_cap = k_tile;
  }
  // the dense-head kernel reads whole 16-byte groups of each 32R-cluster sub-tile
  if (head_r > 0) sh.tile_cap = (int)ceil_div((int64_t)sh.k_tile, 32 * head_r) * 32 * head_r;
  sh.head_r = head_r;
  sh.head_sub = head_r > 0 ? head_sub : 1;
  sh.head_theta = theta;
  const size_t per_warp = ((size_t)sh.tile_cap + 2 * CAND_MAX) * sizeof(float);
  int wmax = (int)std::min<size_t>(kSmemBudget / per_warp, head_r > 0 ? HEAD_MAX_WARPS : 16);
  if (wmax < 1) return false;
  if (head_r > 0 && warps_req > HEAD_MAX_WARPS) return false;
  int warps = warps_req > 0 ? std::min(warps_req, wmax) : std::min(wmax, 8);
  if (warps_req > 0 && (size_t)warps_req * per_warp > kSmemBudget) return false;
  sh.warps = warps;
  sh.tc = tc;
  int bps = assign_max_blocks_per_sm(c->cfg.storage, sh.tile_cap, warps, head_r, sh.head_sub, tc);
  if (bps < 1) return false;
  sh.blocks = bps * c->num_sms;
  *out = sh;
  return true;
}

// Per-(term, tile) offsets for tiles of k_tile clusters: the smallest tile
// in use gives the longest rows, so the buffer only ever grows.
ivf_status ensure_toff(ivf_ctx* c, int k_tile) {
  const int64_t need = c->Dt * (ceil_div(c->kmax, k_tile) + 1);
  if (c->toff && c->toff_len >= need) return IVF_OK;
  dfree(c, c->toff);
  c->toff = nullptr;
  c->toff_len = 0;
  ST(dalloc(c, &c->toff, need));
  c->toff_len = need;
  drop_graphs(c);
  return IVF_OK;
}

// Tensor-core head: a fixed number of dense rows (the GEMM depth, a
// multiple of the 64-slot K-chunk), sized from the lists that qualify now
// with a tenth of room, their transposed copy, and the per-batch buffers;
// lists beyond the rows are read sparsely (exact).
ivf_status setup_tc(ivf_ctx* c, long long wanted) {
  const int64_t vb = (int64_t)storage_bytes(c->cfg.storage);
  const int64_t rows =
      std::min<int64_t>(ceil_div(c->Dt, 64) * 64, std::max<int64_t>(64, ((wanted + wanted / 10) + 63) / 64 * 64));
  if (rows != c->head_max || !c->wdT) {
    dfree(c, c->wd);
    dfree(c, c->wdT);
    c->wd = nullptr;
    c->wdT = nullptr;
    char* p = nullptr;
    ST(dalloc(c, &p, rows * c->kpad * vb));
    c->wd = p;
    char* q = nullptr;
    ST(dalloc(c, &q, rows * c->kpad * vb));
    c->wdT = q;
    c->head_max = rows;
  }
  // batches: GEMM output of at most ~3 GB, a multiple of 128 objects
  c->tc_batch = std::min<int64_t>(c->N, std::max<int64_t>(8192, (int64_t(3) << 30) / (c->kpad * 2)) / 128 * 128);
  if (c->tc_batch < 1) c->tc_batch = c->N;
  if (!c->xh || c->tc_alloc_rows != rows || c->tc_alloc_batch != c->tc_batch || c->tc_alloc_kpad != c->kpad) {
    dfree(c, c->xh);
    dfree(c, c->rho_h);
    dfree(c, c->chunk_nz);
    c->xh = nullptr;
    c->rho_h = nullptr;
    c->chunk_nz = nullptr;
    char* x = nullptr;
    ST(dalloc(c, &x, c->tc_batch * rows * 2));
    c->xh = x;
    char* r = nullptr;
    ST(dalloc(c, &r, c->tc_batch * c->kpad * 2));
    c->rho_h = r;
    ST(dalloc(c, &c->chunk_nz, ceil_div(c->tc_batch, 128) * (rows / 64)));
    c->tc_alloc_rows = rows;
    c->tc_alloc_batch = c->tc_batch;
    c->tc_alloc_kpad = c->kpad;
  }
  return IVF_OK;
}

ivf_status set_shape(ivf_ctx* c, const Shape& sh) {
  if (sh.tiled) ST(ensure_toff(c, sh.k_tile));
  if (sh.tmajor && !c->tcand) {  // kept once allocated (the autotuner switches shapes)
    ST(dalloc(c, &c->tcand, c->N * (int64_t)kTileCand));
    ST(dalloc(c, &c->tcandv, c->N * (int64_t)kTileCand));
    ST(dalloc(c, &c->tcand_n, c->N));
  }
  if (!sh.tc && (c->xh || c->wdT)) {  // the tensor-core buffers are only kept while in use
    CK(c, cudaStreamSynchronize(c->stream));
    dfree(c, c->xh);
    dfree(c, c->rho_h);
    dfree(c, c->chunk_nz);
    dfree(c, c->wdT);
    c->xh = nullptr;
    c->rho_h = nullptr;
    c->chunk_nz = nullptr;
    c->wdT = nullptr;
    c->tc_alloc_rows = c->tc_alloc_batch = c->tc_alloc_kpad = 0;
  }
  c->shape = sh;
  CK(c, assign_prepare(c->cfg.storage, sh.tile_cap, sh.warps, sh.head_r, sh.head_sub, sh.tc));
  if (sh.head_r > 0) ST(alloc_head(c, sh.head_r));
  IvfBuildArgs a = ivf_args(c, c->mcur);
  if (sh.tiled) CK(c, launch_build_toff(a, c->stream));
  if (sh.head_r > 0) {
    CK(c, launch_build_head(a, c->stream));
    long long wanted = 0;
    CK(c, cudaMemcpyAsync(&wanted, &c->dc->heads_wanted, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (sh.tc) {
      ST(setup_tc(c, wanted));
      CK(c, launch_build_head(ivf_args(c, c->mcur), c->stream));  // rows cleared in full for the GEMM
    } else {
      ST(grow_head_if_needed(c, wanted));
    }
  }
  drop_graphs(c);
  return IVF_OK;
}

// One batch of the tensor-core head: dense head values of objects
// [b0, b0 + nb) with their nonzero-chunk flags, then
// rho_h[i][c] = sum_s xh[i][s] * wdT[c][s] on the tensor cores (tc_head.cu:
// FP32 accumulation in TMEM, output in the storage type).
ivf_status enqueue_tc_gemm(ivf_ctx* c, int64_t b0, int64_t nb) {
  CK(c, launch_build_xhead(b0, nb, c->row_ptr, c->term, c->val_store, c->head_slot, c->xh, c->head_max,
                           c->chunk_nz, c->stream));
  TcHeadArgs h;
  h.m = nb;
  h.n = (int32_t)c->kpad;
  h.k = (int32_t)c->head_max;
  h.a = c->xh;
  h.lda = c->head_max;
  h.b = c->wdT;
  h.ldb = c->head_max;
  h.d = c->rho_h;
  h.ldd = c->kpad;
  h.bf16 = c->cfg.storage == IVF_BF16;
  h.out_bf16 = false;  // FP16 product: 2^-11 rounding for either storage type
  h.chunk_nz = c->chunk_nz;
  h.status = &c->dc->status;
  h.num_sms = c->num_sms;
  CK(c, launch_tc_head(h, c->stream));
  return IVF_OK;
}

ivf_status enqueue_main_launches(ivf_ctx* c, const Shape& sh, AssignArgs a);

// Assignment of objects [b0, b0 + nb) with the tensor-core head part.
ivf_status enqueue_tc_batch(ivf_ctx* c, const Shape& sh, int target, int rescore, int64_t b0, int64_t nb,
                            int64_t obj_stride) {
  ST(enqueue_tc_gemm(c, b0, nb));
  CK(c, cudaMemsetAsync(&c->dc->work, 0, sizeof(unsigned long long), c->stream));
  AssignArgs a = assign_args(c, sh, target, rescore);
  a.rho_head = c->rho_h;
  a.rho_ld = c->kpad;
  a.obj_base = b0;
  a.obj_stride = (int32_t)obj_stride;
  a.n_docs = (nb + obj_stride - 1) / obj_stride;
  ST(enqueue_main_launches(c, sh, a));
  return IVF_OK;
}

// The assignment launches of shape sh over a (the main path: every object,
// or a strided sample of them).  Tile-major shapes launch once per tile with
// the (best, id, second) carry in best / assign / gap, then, when a.rescore,
// run the object-major kernel over the near-ties the sweep found, which
// collects their candidate clusters (same arithmetic, so the same bits) and
// queues them for the FP64 re-score.
ivf_status enqueue_main_launches(ivf_ctx* c, const Shape& sh, AssignArgs a) {
  if (!sh.tmajor) {
    CK(c, launch_assign(a, sh.warps, sh.blocks, c->stream, sh.head_r));
    return IVF_OK;
  }
  const int n_tiles = (int)ceil_div(c->kmax, sh.k_tile);
  if (n_tiles > kMaxTileLaunches) return fail(c, IVF_E_UNSUPPORTED, "too many tiles for a tile-major sweep");
  CK(c, cudaMemsetAsync(c->dc->work_tile, 0, sizeof(unsigned long long) * n_tiles, c->stream));
  CK(c, cudaMemsetAsync(&c->dc->n_preflag, 0, sizeof(unsigned int), c->stream));
  const int rescore = a.rescore;
  for (int t = 0; t < n_tiles; ++t) {
    AssignArgs at = a;
    at.tile_lo = t;
    at.tile_hi = t + 1;
    at.work = &c->dc->work_tile[t];
    at.preflag = c->preflag;
    at.n_preflag = &c->dc->n_preflag;
    if (rescore && c->tcand) {
      at.tcand = c->tcand;
      at.tcandv = c->tcandv;
      at.tcand_n = c->tcand_n;
      at.tcand_cap = kTileCand;
    }
    CK(c, launch_assign(at, sh.warps, sh.blocks, c->stream, sh.head_r));
  }
  if (rescore) {
    AssignArgs ar = a;
    ar.obj_list = c->preflag;
    ar.obj_list_n = &c->dc->n_preflag;
    ar.obj_stride = 1;
    ar.work = &c->dc->work_re;
    ar.entries = &c->dc->entries_re;
    ar.n_zero_sim = nullptr;
    CK(c, cudaMemsetAsync(&c->dc->work_re, 0, sizeof(unsigned long long), c->stream));
    CK(c, launch_assign(ar, sh.warps, sh.blocks, c->stream, sh.head_r));
  }
  return IVF_OK;
}

// Work items of class q (q < 0: every object in order) for an assignment launch.
void set_class_objs(ivf_ctx* c, AssignArgs& a, int q) {
  if (q < 0) return;
  const ivf_ctx::ClassPlan& p = c->cls[q];
  a.obj_inst = p.d_inst;
  a.obj_prefix = p.d_prefix;
  a.n_obj_inst = (int32_t)p.insts.size();
  a.n_docs = p.n_objs;
  a.work = &c->dc->work_cls[q];
}

// Device time of one assignment (no re-score) with shape sh over class q's
// objects (q < 0: all): large sets are timed on every s-th object (s <= 16,
// at least 65,536 objects), a sample that spans every instance.
ivf_status time_shape(ivf_ctx* c, const Shape& sh, int q, float* ms_out) {
  const int target = c->alatest < 0 ? 0 : (c->alatest ^ 1);
  if (sh.tc) {
    // the first batch in full (the GEMM works on whole batches): time per object
    const int64_t nb = std::min<int64_t>(c->tc_batch, c->N);
    float ms_min = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      CK(c, cudaMemsetAsync(c->dc, 0, offsetof(DevCounters, status), c->stream));
      CK(c, cudaEventRecord(c->ev[0], c->stream));
      ST(enqueue_tc_batch(c, sh, target, c->cfg.rescore, 0, nb, 1));
      CK(c, cudaEventRecord(c->ev[1], c->stream));
      CK(c, cudaEventSynchronize(c->ev[1]));
      float ms = 0.f;
      CK(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
      ms_min = std::min(ms_min, ms);
    }
    *ms_out = ms_min / (float)nb;
    return IVF_OK;
  }
  // with the re-score on, the candidate bookkeeping (and a tile-major
  // sweep's pass over the near-ties) is part of what is timed
  AssignArgs a = assign_args(c, sh, target, c->cfg.rescore);
  set_class_objs(c, a, q);
  const int64_t n = a.n_docs;
  const int64_t stride = std::max<int64_t>(1, std::min<int64_t>(16, n >> 16));
  a.obj_stride = (int32_t)stride;
  a.n_docs = (n + stride - 1) / stride;
  float ms_min = 1e30f;
  for (int rep = 0; rep < 2; ++rep) {
    CK(c, cudaMemsetAsync(c->dc, 0, offsetof(DevCounters, status), c->stream));
    CK(c, cudaEventRecord(c->ev[0], c->stream));
    if (q < 0)
      ST(enqueue_main_launches(c, sh, a));
    else
      CK(c, launch_assign(a, sh.warps, sh.blocks, c->stream, sh.head_r));
    CK(c, cudaEventRecord(c->ev[1], c->stream));
    CK(c, cudaEventSynchronize(c->ev[1]));
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    ms_min = std::min(ms_min, ms);
  }
  *ms_out = ms_min / (float)a.n_docs;  // per object: comparable across sample sizes
  return IVF_OK;
}

// Kernels for the classes below the last one: untiled (their K fits one
// tile), the sparse kernel or a dense-head kernel reading the rows built for
// the main shape (same theta; the rows are padded to 1,024 clusters).
ivf_status tune_classes(ivf_ctx* c) {
  for (size_t q = 0; q + 1 < c->cls.size(); ++q) {
    ivf_ctx::ClassPlan& p = c->cls[q];
    std::vector<Shape> cands;
    Shape sh;
    const bool no_head = (c->cfg.flags & IVF_FLAG_SPARSE_ONLY) != 0 || c->shape.head_r == 0;
    const bool head_only = (c->cfg.flags & IVF_FLAG_DENSE_HEAD) != 0 && c->shape.head_r > 0;
    if (!head_only && shape_for(c, p.kmax, 0, 0, &sh) && !sh.tiled) cands.push_back(sh);
    if (!no_head) {
      for (int hr : {HEAD_R_SMALL, HEAD_R_MID, HEAD_R_LARGE})
        for (int wp : {8, 4}) {
          if (c->kpad % (32 * hr) != 0) continue;
          if (shape_for(c, p.kmax, 0, wp, &sh, hr, c->shape.head_theta) && !sh.tiled) cands.push_back(sh);
        }
      // K above one register tile: 2,048-cluster shared-memory tiles of
      // 2 x 1,024 or 4 x 512 register sub-tiles
      for (int wp : {4, 8}) {
        if (shape_for(c, p.kmax, 0, wp, &sh, HEAD_R_LARGE, c->shape.head_theta, 2) && !sh.tiled) cands.push_back(sh);
        if (shape_for(c, p.kmax, 0, wp, &sh, HEAD_R_MID, c->shape.head_theta, 4) && !sh.tiled) cands.push_back(sh);
      }
    }
    if (cands.empty()) cands.push_back(c->shape);  // no untiled shape fits: the main class's kernel
    Shape best = cands[0];
    float best_ms = 1e30f;
    for (const Shape& cand : cands) {
      CK(c, assign_prepare(c->cfg.storage, cand.tile_cap, cand.warps, cand.head_r, cand.head_sub));
      float ms = 0.f;
      ST(time_shape(c, cand, (int)q, &ms));
      if (ms < best_ms) {
        best_ms = ms;
        best = cand;
      }
    }
    CK(c, assign_prepare(c->cfg.storage, best.tile_cap, best.warps, best.head_r, best.head_sub));
    p.shape = best;
  }
  c->cls.back().shape = c->shape;
  drop_graphs(c);
  return IVF_OK;
}

// The first choice is made on the initial means (single documents: short
// posting lists); the lists of updated means are far denser, which favours
// other kernels, so the choice is made once more on the first assignment
// after an update step.
// The means keep densifying over the first iterations, so the choice is
// also remade (up to four choices in all) whenever the inverted file has
// grown by more than a third since the last one.
// (IVFD: its object inverted file is rebuilt here after the objects change.)
bool needs_tuning(const ivf_ctx* c) {
  return !c->tuned || (!c->tuned_on_updated_means && c->iteration > 0) ||
         (c->iteration > 0 && c->tunings < 4 && 3 * c->e_cur > 4 * c->e_tuned) ||
         ((c->cfg.flags & IVF_FLAG_IVFD) && !c->ivfd_built);
}

ivf_status autotune(ivf_ctx* c) {
  // IVFD: the object inverted file, and (below) a sparse object-major IVF
  // shape for the pass that collects the near-ties' candidates
  const bool ivfd = (c->cfg.flags & IVF_FLAG_IVFD) != 0;
  if (ivfd) ST(ensure_ivfd(c));
  std::vector<Shape> cands;
  Shape sh;
  if (c->cfg.k_tile > 0) {
    bool ok;
    if (c->cfg.flags & IVF_FLAG_TENSOR_HEAD) {
      ok = c->cfg.storage != IVF_F32 && c->n_inst == 1 && c->cfg.k_tile % (32 * HEAD_R_LARGE) == 0 &&
           shape_for(c, c->kmax, 0, c->cfg.warps_per_block, &sh, HEAD_R_LARGE, 0.25f,
                     c->cfg.k_tile / (32 * HEAD_R_LARGE), true);
    } else if (c->cfg.flags & IVF_FLAG_DENSE_HEAD) {
      const int hr = c->cfg.k_tile < 32 * HEAD_R_LARGE ? HEAD_R_MID : HEAD_R_LARGE;
      ok = c->cfg.k_tile % (32 * hr) == 0 &&
           shape_for(c, c->kmax, 0, c->cfg.warps_per_block, &sh, hr, 0.25f, c->cfg.k_tile / (32 * hr));
    } else {
      ok = shape_for(c, c->kmax, c->cfg.k_tile, c->cfg.warps_per_block, &sh);
    }
    if (!ok) return fail(c, IVF_E_INVALID, "k_tile / warps_per_block not usable for this problem");
    cands.push_back(sh);
  } else {
    const bool tc_only = (c->cfg.flags & IVF_FLAG_TENSOR_HEAD) != 0;
    const bool head_only = (c->cfg.flags & IVF_FLAG_DENSE_HEAD) != 0 || tc_only;
    const bool no_head = (c->cfg.flags & IVF_FLAG_SPARSE_ONLY) != 0 || ivfd;
    // tensor-core head: 16-bit storage, one instance, K over one 1,024-cluster tile
    const bool tc_ok = !no_head && c->cfg.storage != IVF_F32 && c->n_inst == 1 && c->kmax > 32 * HEAD_R_LARGE;
    if (tc_ok && (tc_only || !(c->cfg.flags & IVF_FLAG_DENSE_HEAD)))  // DENSE_HEAD: the CUDA-core head
      // shared-memory tiles of 1-8 head sub-tiles: wider tiles read each
      // object's terms and their list offsets in fewer passes, at fewer
      // resident warps
      for (int sub : {1, 2, 4, 8})
        for (float theta : {0.5f, 0.25f, 0.125f, 0.0625f})
          for (int wp : {4, 8})
            if (shape_for(c, c->kmax, 0, wp, &sh, HEAD_R_LARGE, theta, sub, true)) cands.push_back(sh);
    if (tc_only && !tc_ok) return fail(c, IVF_E_UNSUPPORTED, "the tensor-core head needs FP16/BF16 storage, one instance and K > 1,024");
    if (!head_only) {
      if (shape_for(c, c->kmax, 0, c->cfg.warps_per_block, &sh)) cands.push_back(sh);
      for (int t : kTileChoices)
        if (t < c->kmax && shape_for(c, c->kmax, t, c->cfg.warps_per_block, &sh)) cands.push_back(sh);
    }
    // dense-head kernels (the IFN form for lists covering >= theta K clusters)
    // 512- and 1,024-cluster tiles (fewer registers and more warps per SM
    // against fewer passes over the object's terms); 4-warp blocks fit more
    // warps per SM than 8-warp blocks at ~96 registers
    std::vector<int> rs;
    if (c->kmax <= 32 * HEAD_R_SMALL)
      rs = {HEAD_R_SMALL};
    else
      rs = {HEAD_R_MID, HEAD_R_LARGE};
    if (!no_head && !tc_only) {
      for (int hr : rs)
        for (float theta : {0.5f, 0.25f})
          for (int wp : {8, 4}) {
            if (c->cfg.warps_per_block > 0 && wp != c->cfg.warps_per_block) continue;
            if (hr != HEAD_R_LARGE && wp != 8) continue;
            if (shape_for(c, c->kmax, 0, wp, &sh, hr, theta)) cands.push_back(sh);
          }
      // wider shared-memory tiles for the sparse lists (fewer, longer
      // per-tile slices when K spans many head sub-tiles)
      for (int sub : {2, 4})
        for (float theta : {0.25f, 0.125f})
          for (int wp : {4, 8}) {
            if (c->cfg.warps_per_block > 0 && wp != c->cfg.warps_per_block) continue;
            if (theta < 0.25f && wp != 4) continue;
            if (shape_for(c, c->kmax, 0, wp, &sh, HEAD_R_LARGE, theta, sub)) cands.push_back(sh);
          }
      // 512-cluster register tiles under a 2,048-cluster shared-memory tile:
      // fewer registers (more resident warps) for more passes over the rows
      for (float theta : {0.25f, 0.125f})
        for (int wp : {4, 8}) {
          if (c->cfg.warps_per_block > 0 && wp != c->cfg.warps_per_block) continue;
          if (shape_for(c, c->kmax, 0, wp, &sh, HEAD_R_MID, theta, 4)) cands.push_back(sh);
        }
    }
  }
  // Tile-major twins of the tiled shapes (single-instance contexts; with the
  // tensor-core head, tile-major within each batch of objects):
  // IVF_FLAG_TILE_MAJOR keeps only those, IVF_FLAG_OBJECT_MAJOR none of them.
  {
    const bool only_t = (c->cfg.flags & IVF_FLAG_TILE_MAJOR) != 0 && !ivfd;
    const bool no_t = (c->cfg.flags & IVF_FLAG_OBJECT_MAJOR) != 0 || ivfd;
    std::vector<Shape> with_t;
    for (const Shape& s0 : cands) {
      const bool can = s0.tiled && !c->use_classes && ceil_div(c->kmax, s0.k_tile) <= kMaxTileLaunches;
      if (!only_t || !can) {
        if (!only_t) with_t.push_back(s0);
      }
      if (can && !no_t) {
        Shape s1 = s0;
        s1.tmajor = true;
        with_t.push_back(s1);
      }
    }
    if (only_t && with_t.empty()) return fail(c, IVF_E_UNSUPPORTED, "no tiled shape for a tile-major sweep");
    cands.swap(with_t);
  }
  if (cands.empty()) return fail(c, IVF_E_UNSUPPORTED, "no accumulator tile fits shared memory");
  // Contexts of the same shape in one process reuse the first choice, so
  // their FP32 rounding (which depends on the kernel family) is the same.
  const int kflags = (int)(c->cfg.flags & (IVF_FLAG_DENSE_HEAD | IVF_FLAG_SPARSE_ONLY | IVF_FLAG_TENSOR_HEAD |
                                           IVF_FLAG_TILE_MAJOR | IVF_FLAG_OBJECT_MAJOR));
  auto key = std::make_tuple(c->N >> 12, (int64_t)c->kmax, c->Dt >> 12,
                             (c->cfg.storage * 256 + kflags) * 8 + std::min(c->tunings, 7),
                             c->n_inst);
  const bool cacheable = c->cfg.k_tile == 0 && c->cfg.warps_per_block == 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && cacheable) {
      ST(set_shape(c, it->second.main));
      for (size_t q = 0; q + 1 < c->cls.size() && q < it->second.cls.size(); ++q) c->cls[q].shape = it->second.cls[q];
      if (!c->cls.empty()) c->cls.back().shape = c->shape;
      c->tuned = true;
      c->tuned_on_updated_means = c->iteration > 0;
      c->e_tuned = c->e_cur;
      ++c->tunings;
      return IVF_OK;
    }
  }
  const int main_q = c->use_classes ? (int)c->cls.size() - 1 : -1;
  Shape best_sh = cands[0];
  if (cands.size() > 1) {
    // Time one assignment per candidate (no re-score) on the real data.
    float best_ms = 1e30f;
    for (const Shape& cand : cands) {
      ST(set_shape(c, cand));
      float ms = 0.f;
      ST(time_shape(c, cand, main_q, &ms));
      if (ms < best_ms) {
        best_ms = ms;
        best_sh = cand;
      }
    }
  }
  ST(set_shape(c, best_sh));
  if (c->use_classes) ST(tune_classes(c));
  c->tuned = true;
  c->tuned_on_updated_means = c->iteration > 0;
  c->e_tuned = c->e_cur;
  ++c->tunings;
  if (cacheable) {
    TuneChoice tc;
    tc.main = best_sh;
    for (size_t q = 0; q + 1 < c->cls.size(); ++q) tc.cls.push_back(c->cls[q].shape);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = tc;
  }
  return IVF_OK;
}

// ------------------------------------------------------ enqueue phases

cudaError_t timing_event(ivf_ctx* c, size_t* idx) {
  if (c->tev_used == c->tev.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->tev.push_back(e);
  }
  *idx = c->tev_used++;
  return cudaEventRecord(c->tev[*idx], c->stream);
}

// Assignment (+ re-score + reductions) into buffer `target`, previous `prev` (-1 none).
ivf_status enqueue_assign(ivf_ctx* c, int target, int prev, bool timed = false) {
  cudaStream_t s = c->stream;
  CK(c, cudaMemsetAsync(c->dc, 0, offsetof(DevCounters, status), s));
  CK(c, cudaMemsetAsync(c->inst_changed, 0, sizeof(long long) * c->n_inst, s));
  size_t e0 = 0, e1 = 0, e2 = 0;
  if (timed) CK(c, timing_event(c, &e0));
  if (c->cfg.flags & IVF_FLAG_IVFD) {
    CK(c, cudaMemsetAsync(&c->dc->n_preflag, 0, sizeof(unsigned int), s));
    CK(c, launch_assign_ivfd(ivfd_args(c, target, c->cfg.rescore), s));
    if (c->cfg.rescore) {  // the near-ties' candidates, from the IVF kernel (same sums)
      AssignArgs ar = assign_args(c, c->shape, target, 1);
      ar.obj_list = c->preflag;
      ar.obj_list_n = &c->dc->n_preflag;
      ar.work = &c->dc->work_re;
      ar.entries = &c->dc->entries_re;
      ar.n_zero_sim = nullptr;
      CK(c, cudaMemsetAsync(&c->dc->work_re, 0, sizeof(unsigned long long), s));
      CK(c, launch_assign(ar, c->shape.warps, c->shape.blocks, s, c->shape.head_r));
    }
  } else if (c->use_classes) {
    // one launch per class of instances, each with the kernel chosen for it
    for (size_t q = 0; q < c->cls.size(); ++q) {
      const Shape& sh = c->cls[q].shape;
      AssignArgs a = assign_args(c, sh, target, c->cfg.rescore);
      set_class_objs(c, a, (int)q);
      CK(c, launch_assign(a, sh.warps, sh.blocks, s, sh.head_r));
    }
  } else if (c->shape.tc) {
    for (int64_t b0 = 0; b0 < c->N; b0 += c->tc_batch)
      ST(enqueue_tc_batch(c, c->shape, target, c->cfg.rescore, b0, std::min<int64_t>(c->tc_batch, c->N - b0), 1));
  } else {
    ST(enqueue_main_launches(c, c->shape, assign_args(c, c->shape, target, c->cfg.rescore)));
  }
  if (timed) CK(c, timing_event(c, &e1));
  if (c->cfg.rescore) {
    RescoreArgs r{};
    r.row_ptr = c->row_ptr;
    r.term = c->term;
    r.val32 = c->val32;
    r.n_inst = c->n_inst;
    r.inst_docs = c->inst_docs;
    r.inst_clu = c->inst_clu;
    r.mptr = c->mptr[c->mcur];
    r.mterm = c->mterm[c->mcur];
    r.mval = c->mval[c->mcur];
    r.n_flagged = &c->dc->n_flagged;
    r.flag_obj = c->flag_obj;
    r.flag_cnt = c->flag_cnt;
    r.flag_cand = c->flag_cand;
    r.assign = c->assign[target];
    r.best = c->best;
    r.gap = c->gap;
    r.err = c->errb;
    r.nx = c->nx;
    r.n_rescored = &c->dc->n_rescored;
    // one warp per flagged object, latency bound: a full GPU of warps (8
    // blocks of 8 warps per SM) keeps enough FP64 dot products in flight
    CK(c, launch_rescore(r, 8 * c->num_sms, s));
  }
  ReduceArgs ra{};
  ra.n_docs = c->N;
  ra.assign = c->assign[target];
  ra.prev = prev >= 0 ? c->assign[prev] : nullptr;
  ra.best = c->best;
  ra.n_inst = c->n_inst;
  ra.inst_docs = c->inst_docs;
  ra.inst_changed = c->inst_changed;
  ra.part_obj = c->part_obj;
  ra.part_cnt = c->part_cnt;
  ra.out_obj = &c->dc->objective;
  ra.out_cnt = c->dc->cnt;
  ra.zero_sim = &c->dc->zero_sim;
  ra.entries = &c->dc->entries;
  ra.n_rescored = &c->dc->n_rescored;
  ra.acc_entries = &c->dc->acc_entries;
  ra.acc_rescored = &c->dc->acc_rescored;
  CK(c, launch_reduce(ra, c->red_blocks, s));
  if (timed) {
    CK(c, timing_event(c, &e2));
    (void)e1;
    (void)e2;
    c->tcalls.push_back({0, e0});
  }
  return IVF_OK;
}

// Everything the update kernels read and write, from assignment buffer src:
// means mcur -> mcur^1.
UpdateArgs update_args(ivf_ctx* c, int src) {
  const int mo = c->mcur, mn = c->mcur ^ 1;
  UpdateArgs u{};
  u.n_docs = c->N;
  u.nnz = c->nnz;
  u.n_inst = c->n_inst;
  u.kt = c->Kt;
  u.dt = c->Dt;
  u.tbits = c->tbits_local;
  u.kbits = c->kbits;
  u.inst_toff = c->inst_toff;
  u.row_ptr = c->row_ptr;
  u.term = c->term;
  u.val32 = c->val32;
  u.inst_docs = c->inst_docs;
  u.inst_clu = c->inst_clu;
  u.assign = c->assign[src];
  u.zterm = c->zterm;
  u.zov = c->zov;
  u.empty_policy = c->cfg.empty_policy;
  u.mptr_old = c->mptr[mo];
  u.mterm_old = c->mterm[mo];
  u.mval_old = c->mval[mo];
  u.mptr_new = c->mptr[mn];
  u.mterm_new = c->mterm[mn];
  u.mval_new = c->mval[mn];
  u.mclu_new = c->mclu[mn];
  u.cap = c->cap;
  u.cl_ptr = c->cl_ptr;
  u.members = c->members;
  u.sum_norm = c->sum_norm;
  u.rnorm = c->rnorm;
  u.k64a = c->k64a;
  u.k64b = c->k64b;
  u.v32a = c->v32a;
  u.v32b = c->v32b;
  u.flags = c->flags;
  u.starts = c->starts;
  u.ukey = c->ukey;
  u.usum = c->usum;
  u.uptr = c->uptr;
  u.newlen = c->newlen;
  u.zrun = c->zrun;
  u.d_nnz = c->d_nnz;
  u.d_n = c->d_n;
  u.d_u = c->d_u;
  u.temp = c->temp;
  u.status = &c->dc->status;
  u.means_negative = &c->dc->means_negative[mn];
  return u;
}

// Update from assignment buffer `src`: means mcur -> mcur^1, then the inverted file.
ivf_status enqueue_update(ivf_ctx* c, int src) {
  UpdateArgs u = update_args(c, src);
  CK(c, cudaMemsetAsync(u.means_negative, 0, sizeof(unsigned), c->stream));
  CK(c, launch_update_means(u, c->stream));
  ST(enqueue_build_ivf(c, c->mcur ^ 1));
  return IVF_OK;
}

// Run buffers (flags, starts, ukey, usum) and sort scratch for n run sums.
ivf_status ensure_runs(ivf_ctx* c, int64_t n) {
  if (n > c->run_cap) {
    void* olds[] = {c->flags, c->starts, c->ukey, c->usum};
    for (void* p : olds) dfree(c, p);
    c->flags = nullptr;
    c->starts = nullptr;
    c->ukey = nullptr;
    c->usum = nullptr;
    ST(dalloc(c, &c->flags, n + 1));
    ST(dalloc(c, &c->starts, n + 1));
    ST(dalloc(c, &c->ukey, n));
    ST(dalloc(c, &c->usum, n));
    c->run_cap = n;
    drop_graphs(c);
  }
  if (n > c->scratch_len) ST(alloc_scratch(c, n));
  return IVF_OK;
}

// Update from the member sums in part_* (gathered from shards): means
// mcur -> mcur^1, then the inverted file.
ivf_status enqueue_update_from_partials(ivf_ctx* c) {
  UpdateArgs u = update_args(c, c->alatest >= 0 ? c->alatest : 0);
  PartialArgs p{};
  p.n_max = std::max<int64_t>(1, c->part_n);
  p.d_n = c->d_part_n;
  p.cluster = c->part_cluster;
  p.term = c->part_term;
  p.sum = c->part_sum;
  CK(c, cudaMemsetAsync(u.means_negative, 0, sizeof(unsigned), c->stream));
  CK(c, launch_update_from_partials(u, p, c->stream));
  ST(enqueue_build_ivf(c, c->mcur ^ 1));
  return IVF_OK;
}

void fill_stats(ivf_ctx* c, ivf_iter_stats* st) {
  const DevCounters& h = *c->hc;
  c->e_cur = h.ivf_e;
  st->n_changed = (int64_t)h.cnt[0];
  st->n_zero_sim = (int64_t)h.cnt[1];
  st->entries_visited = (int64_t)h.entries;
  st->ivf_entries = c->e_cur;
  st->n_flagged = (int64_t)h.n_flagged;
  st->n_rescored = (int64_t)h.n_rescored;
  st->objective = h.objective;
  st->t_assign_ms = 0.f;
  st->t_update_ms = 0.f;
}

ivf_status read_counters(ivf_ctx* c) {
  CK(c, cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->e_cur = c->hc->ivf_e;
  return IVF_OK;
}

ivf_status copy_mean_rows_in(ivf_ctx* c, const int64_t* mean_ptr, std::vector<int64_t>* hp) {
  hp->resize(c->Kt + 1);
  CK(c, cudaMemcpy(hp->data(), mean_ptr, sizeof(int64_t) * (c->Kt + 1), cudaMemcpyDefault));
  if ((*hp)[0] != 0) return fail(c, IVF_E_INVALID, "mean_ptr[0] must be 0");
  for (int64_t j = 0; j < c->Kt; ++j)
    if ((*hp)[j + 1] < (*hp)[j]) return fail(c, IVF_E_INVALID, "mean_ptr must be non-decreasing");
  return IVF_OK;
}

// Grow the means / inverted-file arrays to new_cap entries, keeping the
// current means (buffer mcur), which an update step still reads.
ivf_status grow_means(ivf_ctx* c, int64_t new_cap) {
  const int mb = c->mcur;
  int64_t e_old = 0;
  CK(c, cudaMemcpyAsync(&e_old, c->mptr[mb] + c->Kt, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  int32_t* t_keep = nullptr;
  double* v_keep = nullptr;
  int32_t* cl_keep = nullptr;
  ST(dalloc(c, &t_keep, new_cap));
  ST(dalloc(c, &v_keep, new_cap));
  ST(dalloc(c, &cl_keep, new_cap));
  CK(c, cudaMemcpyAsync(t_keep, c->mterm[mb], sizeof(int32_t) * e_old, cudaMemcpyDeviceToDevice, c->stream));
  CK(c, cudaMemcpyAsync(v_keep, c->mval[mb], sizeof(double) * e_old, cudaMemcpyDeviceToDevice, c->stream));
  CK(c, cudaMemcpyAsync(cl_keep, c->mclu[mb], sizeof(int32_t) * e_old, cudaMemcpyDeviceToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  void* old[] = {c->mterm[0], c->mterm[1], c->mval[0], c->mval[1], c->mclu[0], c->mclu[1], c->cid16, c->cid32, c->w};
  for (void* p : old) dfree(c, p);
  c->mterm[mb] = t_keep;
  c->mval[mb] = v_keep;
  c->mclu[mb] = cl_keep;
  ST(dalloc(c, &c->mterm[mb ^ 1], new_cap));
  ST(dalloc(c, &c->mval[mb ^ 1], new_cap));
  ST(dalloc(c, &c->mclu[mb ^ 1], new_cap));
  ST(dalloc(c, &c->cid16, new_cap + 8));
  ST(dalloc(c, &c->cid32, new_cap));
  char* wp = nullptr;
  ST(dalloc(c, &wp, (new_cap + 8) * (int64_t)storage_bytes(c->cfg.storage)));
  c->w = wp;
  c->cap = new_cap;
  if (std::max<int64_t>({c->nnz, c->cap, c->N + 1}) > c->scratch_len)
    ST(alloc_scratch(c, std::max<int64_t>({c->nnz, c->cap, c->N + 1})));
  drop_graphs(c);
  return IVF_OK;
}

// After an update step (means mcur -> mcur^1) whose new means did not fit
// (STS_CAPACITY): grow and run the update again from the same assignment.
// Synchronises.
// heads_wanted (optional) receives the number of lists that qualified as
// dense rows in the rebuilt inverted file, read in the same synchronisation.
ivf_status redo_update_if_overflow(ivf_ctx* c, int src, long long* heads_wanted = nullptr,
                                   bool from_partials = false) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    unsigned st = 0;
    int64_t e_new = 0;
    CK(c, cudaMemcpyAsync(&st, &c->dc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&e_new, c->mptr[c->mcur ^ 1] + c->Kt, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    if (heads_wanted)
      CK(c, cudaMemcpyAsync(heads_wanted, &c->dc->heads_wanted, sizeof(long long), cudaMemcpyDeviceToHost,
                            c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (st & STS_TIMEOUT) return check_status(c);
    if (!(st & STS_CAPACITY)) {
      c->e_cur = e_new;
      return IVF_OK;
    }
    CK(c, cudaMemsetAsync(&c->dc->status, 0, sizeof(unsigned), c->stream));
    ST(grow_means(c, e_new + e_new / 4 + 4096));
    if (from_partials)
      ST(enqueue_update_from_partials(c));
    else
      ST(enqueue_update(c, src));
  }
  return fail(c, IVF_E_OOM, "new means exceed the inverted-file capacity after growing it");
}

ivf_status ensure_capacity(ivf_ctx* c, int64_t e0) {
  if (e0 <= c->cap) return IVF_OK;
  ST(alloc_means(c, e0 + e0 / 4 + 4096));  // later updates grow it on demand
  ST(alloc_scratch(c, std::max<int64_t>({c->nnz, c->cap, c->N + 1})));
  c->means_set = false;
  return IVF_OK;
}

ivf_status finish_set_means(ivf_ctx* c) {
  ST(check_status(c));
  // tile offsets need term_ptr, so the first build may precede the shape choice
  ST(enqueue_build_ivf(c, c->mcur));
  ST(read_counters(c));
  ST(check_status(c));
  c->means_set = true;
  c->alatest = -1;
  c->iteration = 0;
  // new means: the kernel is chosen again (a cached choice for this shape
  // is taken as is), so a context follows the same kernel sequence as a
  // fresh one given the same data
  c->tuned = false;
  c->tuned_on_updated_means = false;
  c->tunings = 0;
  c->e_tuned = 0;
  c->members_valid = false;
  drop_graphs(c);
  return IVF_OK;
}

// One full iteration (assign + update) enqueued on the stream.
ivf_status enqueue_iteration(ivf_ctx* c, int target, int prev) {
  ST(enqueue_assign(c, target, prev));
  ST(enqueue_update(c, target));
  CK(c, cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream));
  return IVF_OK;
}

}  // namespace

// ================================================================= C ABI

extern "C" {

const char* ivf_version(void) { return "libivfkm 0.1 (sm_103a)"; }

int64_t ivf_launch_count(void) { return (int64_t)g_launches.load(); }

const char* ivf_last_error(const ivf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void ivf_destroy(ivf_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  for (cudaEvent_t ev : {ctx->ev_src, ctx->ev_staged, ctx->ev_staging_free})
    if (ev) cudaEventDestroy(ev);
  drop_graphs(ctx);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  for (auto& ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : ctx->tev) cudaEventDestroy(ev);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->hc) cudaFreeHost(ctx->hc);
  delete ctx;
}

ivf_status ivf_create(const ivf_config* cfg, const int64_t* row_ptr, const int32_t* term, const float* val,
                      void* cuda_stream, ivf_ctx** out) {
  if (!out) return IVF_E_INVALID;
  *out = nullptr;
  if (validate_cfg(cfg) != IVF_OK || !row_ptr || (!term && cfg->nnz > 0) || (!val && cfg->nnz > 0))
    return IVF_E_INVALID;
  if (cfg->n_docs < 1 || cfg->n_terms < 1 || cfg->k < 1 || cfg->k > cfg->n_docs || cfg->nnz < 0)
    return IVF_E_INVALID;
  std::vector<int64_t> docs = {0, cfg->n_docs};
  std::vector<int32_t> terms = {(int32_t)cfg->n_terms};
  std::vector<int32_t> ks = {cfg->k};
  if (cfg->n_terms >= (int64_t(1) << 31)) return IVF_E_UNSUPPORTED;
  return create_common(cfg, 1, docs, terms, ks, row_ptr, term, val, cuda_stream, out);
}

ivf_status ivfb_create(const ivf_config* cfg, int32_t n_inst, const int64_t* inst_docs, const int32_t* inst_terms,
                       const int32_t* inst_k, const int64_t* row_ptr, const int32_t* term, const float* val,
                       void* cuda_stream, ivf_ctx** out) {
  if (!out) return IVF_E_INVALID;
  *out = nullptr;
  if (validate_cfg(cfg) != IVF_OK || n_inst < 1 || !inst_docs || !inst_terms || !inst_k || !row_ptr)
    return IVF_E_INVALID;
  if (cfg->flags & IVF_FLAG_IVFD) return IVF_E_UNSUPPORTED;
  std::vector<int64_t> docs(n_inst + 1);
  std::vector<int32_t> terms(n_inst), ks(n_inst);
  if (cudaMemcpy(docs.data(), inst_docs, sizeof(int64_t) * (n_inst + 1), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(terms.data(), inst_terms, sizeof(int32_t) * n_inst, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(ks.data(), inst_k, sizeof(int32_t) * n_inst, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return IVF_E_INVALID;
  }
  if (docs[0] != 0) return IVF_E_INVALID;
  for (int b = 0; b < n_inst; ++b) {
    const int64_t nb = docs[b + 1] - docs[b];
    if (nb < 1 || terms[b] < 1 || ks[b] < 1 || ks[b] > nb) return IVF_E_INVALID;
  }
  ivf_config c2 = *cfg;
  c2.nnz = -1;
  return create_common(&c2, n_inst, docs, terms, ks, row_ptr, term, val, cuda_stream, out);
}

ivf_status ivf_load_objects(ivf_ctx* c, const int64_t* row_ptr, const int32_t* term, const float* val) {
  if (!c || !row_ptr || (c->nnz > 0 && (!term || !val))) return fail(c, IVF_E_INVALID, "null argument");
  ST(ensure_staging(c));
  cudaStream_t cs = c->copy_stream;
  c->objects_pending = false;  // a load not yet committed is replaced
  // the staging copy is free once the last commit's device copies ran
  CK(c, cudaStreamWaitEvent(cs, c->ev_staging_free, 0));
  // device sources are read after the work already on the context stream
  if (device_resident(row_ptr) || device_resident(term) || device_resident(val)) {
    CK(c, cudaEventRecord(c->ev_src, c->stream));
    CK(c, cudaStreamWaitEvent(cs, c->ev_src, 0));
  }
  // row_ptr is checked on the device before the big copies are issued: the
  // one synchronisation of this call (on the copy stream only)
  CK(c, cudaMemcpyAsync(c->st_row_ptr, row_ptr, sizeof(int64_t) * (c->N + 1), cudaMemcpyDefault, cs));
  CK(c, cudaMemsetAsync(c->d_load_status, 0, sizeof(unsigned), cs));
  CK(c, launch_check_row_ptr(c->st_row_ptr, c->N, c->nnz, c->d_load_status, cs));
  unsigned st = 0;
  CK(c, cudaMemcpyAsync(&st, c->d_load_status, sizeof(unsigned), cudaMemcpyDeviceToHost, cs));
  CK(c, cudaStreamSynchronize(cs));
  if (st & STS_BAD_ROWS) return fail(c, IVF_E_INVALID, "row_ptr must start at 0, end at nnz and be non-decreasing");
  CK(c, cudaMemcpyAsync(c->st_term, term, sizeof(int32_t) * c->nnz, cudaMemcpyDefault, cs));
  CK(c, cudaMemcpyAsync(c->st_val32, val, sizeof(float) * c->nnz, cudaMemcpyDefault, cs));
  CK(c, cudaEventRecord(c->ev_staged, cs));
  c->objects_pending = true;
  return IVF_OK;
}

ivf_status ivf_set_means(ivf_ctx* c, const int64_t* mean_ptr, const int32_t* mean_term, const float* mean_val) {
  if (!c || !mean_ptr) return fail(c, IVF_E_INVALID, "null argument");
  if (c->n_inst != 1) return fail(c, IVF_E_UNSUPPORTED, "batched contexts take means from documents");
  std::vector<int64_t> hp;
  ST(copy_mean_rows_in(c, mean_ptr, &hp));
  const int64_t e0 = hp[c->Kt];
  if (e0 > 0 && (!mean_term || !mean_val)) return fail(c, IVF_E_INVALID, "null mean arrays");
  ST(ensure_capacity(c, e0));
  const int mb = c->mcur;
  std::vector<float> hv(e0);
  std::vector<double> hd(e0);
  CK(c, cudaMemcpy(hv.data(), mean_val, sizeof(float) * e0, cudaMemcpyDefault));
  for (int64_t e = 0; e < e0; ++e) hd[e] = (double)hv[e];
  CK(c, cudaMemcpyAsync(c->mptr[mb], hp.data(), sizeof(int64_t) * (c->Kt + 1), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->mterm[mb], mean_term, sizeof(int32_t) * e0, cudaMemcpyDefault, c->stream));
  CK(c, cudaMemcpyAsync(c->mval[mb], hd.data(), sizeof(double) * e0, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemsetAsync(&c->dc->means_negative[mb], 0, sizeof(unsigned), c->stream));
  CK(c, launch_normalise_rows(c->Kt, c->mptr[mb], c->mval[mb], c->mclu[mb], c->Dt, c->mterm[mb], &c->dc->status, 1,
                              &c->dc->means_negative[mb], c->stream));
  return finish_set_means(c);
}

ivf_status ivf_restore_means(ivf_ctx* c, const int64_t* ptr, const int32_t* term, const double* val,
                             int32_t iteration) {
  if (!c || !ptr) return fail(c, IVF_E_INVALID, "null argument");
  std::vector<int64_t> hp;
  ST(copy_mean_rows_in(c, ptr, &hp));
  const int64_t e0 = hp[c->Kt];
  if (e0 > 0 && (!term || !val)) return fail(c, IVF_E_INVALID, "null mean arrays");
  ST(ensure_capacity(c, e0));
  const int mb = c->mcur;
  std::vector<int32_t> ht(e0);
  CK(c, cudaMemcpy(ht.data(), term, sizeof(int32_t) * e0, cudaMemcpyDefault));
  if (c->n_inst > 1) {  // local -> global term ids
    for (int64_t j = 0; j < c->Kt; ++j) {
      int b = (int)(std::upper_bound(c->h_inst_clu.begin(), c->h_inst_clu.end(), (int32_t)j) - c->h_inst_clu.begin()) - 1;
      for (int64_t e = hp[j]; e < hp[j + 1]; ++e) ht[e] += (int32_t)c->h_inst_toff[b];
    }
  }
  CK(c, cudaMemcpyAsync(c->mptr[mb], hp.data(), sizeof(int64_t) * (c->Kt + 1), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->mterm[mb], ht.data(), sizeof(int32_t) * e0, cudaMemcpyHostToDevice, c->stream));
  std::vector<double> hv(e0);
  CK(c, cudaMemcpy(hv.data(), val, sizeof(double) * e0, cudaMemcpyDefault));
  CK(c, cudaMemcpyAsync(c->mval[mb], hv.data(), sizeof(double) * e0, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemsetAsync(&c->dc->means_negative[mb], 0, sizeof(unsigned), c->stream));
  CK(c, launch_normalise_rows(c->Kt, c->mptr[mb], c->mval[mb], c->mclu[mb], c->Dt, c->mterm[mb], &c->dc->status, 0,
                              &c->dc->means_negative[mb], c->stream));
  ST(finish_set_means(c));
  c->iteration = iteration;
  return IVF_OK;
}

ivf_status ivf_set_means_from_docs(ivf_ctx* c, const int32_t* doc_ids) {
  if (!c || !doc_ids) return fail(c, IVF_E_INVALID, "null argument");
  ST(commit_objects(c));
  std::vector<int32_t> ids(c->Kt);
  CK(c, cudaMemcpy(ids.data(), doc_ids, sizeof(int32_t) * c->Kt, cudaMemcpyDefault));
  // local -> global object ids; distinct within each instance
  for (int b = 0; b < c->n_inst; ++b) {
    const int64_t nb = c->h_inst_docs[b + 1] - c->h_inst_docs[b];
    std::vector<int32_t> seen(ids.begin() + c->h_inst_clu[b], ids.begin() + c->h_inst_clu[b + 1]);
    std::sort(seen.begin(), seen.end());
    for (size_t q = 0; q < seen.size(); ++q) {
      if (seen[q] < 0 || seen[q] >= nb) return fail(c, IVF_E_INVALID, "doc id out of range");
      if (q && seen[q] == seen[q - 1]) return fail(c, IVF_E_INVALID, "doc ids must be distinct");
    }
    for (int32_t j = c->h_inst_clu[b]; j < c->h_inst_clu[b + 1]; ++j) ids[j] += (int32_t)c->h_inst_docs[b];
  }
  // row lengths on the host to size the means
  std::vector<int64_t> hrp(c->N + 1);
  CK(c, cudaMemcpyAsync(hrp.data(), c->row_ptr, sizeof(int64_t) * (c->N + 1), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  int64_t e0 = 0;
  for (int64_t j = 0; j < c->Kt; ++j) e0 += hrp[ids[j] + 1] - hrp[ids[j]];
  ST(ensure_capacity(c, e0));
  int32_t* d_ids = reinterpret_cast<int32_t*>(c->flag_obj);  // scratch: Kt <= N
  const int mb = c->mcur;
  CK(c, cudaMemcpyAsync(d_ids, ids.data(), sizeof(int32_t) * c->Kt, cudaMemcpyHostToDevice, c->stream));
  CK(c, launch_gather_rows(c->Kt, d_ids, c->row_ptr, c->term, c->val32, c->mptr[mb], c->mterm[mb], c->mval[mb],
                           c->temp, c->stream, 0));
  CK(c, launch_gather_rows(c->Kt, d_ids, c->row_ptr, c->term, c->val32, c->mptr[mb], c->mterm[mb], c->mval[mb],
                           c->temp, c->stream, 1));
  CK(c, cudaMemsetAsync(&c->dc->means_negative[mb], 0, sizeof(unsigned), c->stream));
  CK(c, launch_normalise_rows(c->Kt, c->mptr[mb], c->mval[mb], c->mclu[mb], c->Dt, c->mterm[mb], &c->dc->status, 1,
                              &c->dc->means_negative[mb], c->stream));
  return finish_set_means(c);
}

ivf_status ivf_assign(ivf_ctx* c, int32_t* assign_out, float* best_out, float* gap_out, ivf_iter_stats* stats_out) {
  if (!c) return IVF_E_INVALID;
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  ST(commit_objects(c));
  if (needs_tuning(c)) ST(autotune(c));
  const int target = c->alatest < 0 ? 0 : (c->alatest ^ 1);
  const int prev = c->alatest;
  CK(c, cudaEventRecord(c->ev[0], c->stream));
  ST(enqueue_assign(c, target, prev, c->timing));
  CK(c, cudaEventRecord(c->ev[1], c->stream));
  c->alatest = target;
  if (assign_out)
    CK(c, cudaMemcpyAsync(assign_out, c->assign[target], sizeof(int32_t) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  if (best_out) CK(c, cudaMemcpyAsync(best_out, c->best, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  if (gap_out) CK(c, cudaMemcpyAsync(gap_out, c->gap, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  if (stats_out) {
    ST(read_counters(c));
    if (c->hc->status & STS_TIMEOUT) return check_status(c);
    fill_stats(c, stats_out);
    CK(c, cudaEventElapsedTime(&stats_out->t_assign_ms, c->ev[0], c->ev[1]));
  }
  return IVF_OK;
}

ivf_status ivf_update(ivf_ctx* c) {
  if (!c) return IVF_E_INVALID;
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  if (c->alatest < 0) return fail(c, IVF_E_STATE, "no assignment to update from");
  size_t e0 = 0, e1 = 0;
  if (c->timing) CK(c, timing_event(c, &e0));
  ST(enqueue_update(c, c->alatest));
  if (c->timing) {
    CK(c, timing_event(c, &e1));
    c->tcalls.push_back({1, e0});
  }
  long long wanted = 0;
  ST(redo_update_if_overflow(c, c->alatest, &wanted));
  c->mcur ^= 1;
  c->iteration += 1;
  c->members_valid = true;
  ST(grow_head_if_needed(c, wanted));
  return IVF_OK;
}

ivf_status ivf_get_partial_sums(ivf_ctx* c, int64_t cap, int32_t* cluster, int32_t* term, double* sum,
                                int64_t* n_out) {
  if (!c || !n_out) return fail(c, IVF_E_INVALID, "null argument");
  if (c->n_inst != 1) return fail(c, IVF_E_UNSUPPORTED, "partial sums of a batched context");
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  if (c->alatest < 0) return fail(c, IVF_E_STATE, "no assignment to sum from");
  UpdateArgs u = update_args(c, c->alatest);
  CK(c, launch_member_sums(u, c->stream));
  int64_t n = 0;
  CK(c, cudaMemcpyAsync(&n, c->d_u, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  *n_out = n;
  if (!cluster && !term && !sum) return IVF_OK;
  if (cap < n) return fail(c, IVF_E_INVALID, "output capacity below the number of member sums");
  if (n > c->part_cap) {
    dfree(c, c->part_cluster);
    dfree(c, c->part_term);
    dfree(c, c->part_sum);
    c->part_cluster = nullptr;
    c->part_term = nullptr;
    c->part_sum = nullptr;
    ST(dalloc(c, &c->part_cluster, n));
    ST(dalloc(c, &c->part_term, n));
    ST(dalloc(c, &c->part_sum, n));
    c->part_cap = n;
  }
  CK(c, launch_partial_out(u, std::max<int64_t>(1, n), c->part_cluster, c->part_term, c->part_sum, c->stream));
  if (cluster) CK(c, cudaMemcpyAsync(cluster, c->part_cluster, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream));
  if (term) CK(c, cudaMemcpyAsync(term, c->part_term, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream));
  if (sum) CK(c, cudaMemcpyAsync(sum, c->part_sum, sizeof(double) * n, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return IVF_OK;
}

ivf_status ivf_update_from_partials(ivf_ctx* c, int64_t n_total, const int32_t* cluster, const int32_t* term,
                                    const double* sum) {
  if (!c || n_total < 0 || (n_total > 0 && (!cluster || !term || !sum))) return fail(c, IVF_E_INVALID, "bad arguments");
  if (c->n_inst != 1) return fail(c, IVF_E_UNSUPPORTED, "partial sums of a batched context");
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  if (n_total >= (int64_t(1) << 32) - 2) return fail(c, IVF_E_UNSUPPORTED, "too many member sums");
  ST(ensure_runs(c, std::max<int64_t>(1, n_total)));
  if (n_total > c->part_cap) {
    dfree(c, c->part_cluster);
    dfree(c, c->part_term);
    dfree(c, c->part_sum);
    c->part_cluster = nullptr;
    c->part_term = nullptr;
    c->part_sum = nullptr;
    ST(dalloc(c, &c->part_cluster, n_total));
    ST(dalloc(c, &c->part_term, n_total));
    ST(dalloc(c, &c->part_sum, n_total));
    c->part_cap = n_total;
  }
  if (n_total > 0) {
    CK(c, cudaMemcpyAsync(c->part_cluster, cluster, sizeof(int32_t) * n_total, cudaMemcpyDefault, c->stream));
    CK(c, cudaMemcpyAsync(c->part_term, term, sizeof(int32_t) * n_total, cudaMemcpyDefault, c->stream));
    CK(c, cudaMemcpyAsync(c->part_sum, sum, sizeof(double) * n_total, cudaMemcpyDefault, c->stream));
  }
  // the ids are checked on the device copy before they key a sort
  c->part_n = n_total;
  CK(c, cudaMemcpyAsync(c->d_part_n, &c->part_n, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  CK(c, launch_check_partials(n_total, c->part_cluster, c->part_term, (int32_t)c->Kt, (int32_t)c->Dt,
                              &c->dc->status, c->stream));
  ST(check_status(c));
  ST(enqueue_update_from_partials(c));
  long long wanted = 0;
  ST(redo_update_if_overflow(c, c->alatest, &wanted, true));
  c->mcur ^= 1;
  c->iteration += 1;
  c->members_valid = false;
  ST(grow_head_if_needed(c, wanted));
  return IVF_OK;
}

ivf_status ivf_iterate(ivf_ctx* c, int32_t max_iter, int32_t* iters_done, int32_t* converged,
                       ivf_iter_stats* last_stats) {
  if (!c) return IVF_E_INVALID;
  if (max_iter < 0) return fail(c, IVF_E_INVALID, "max_iter < 0");
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  ST(commit_objects(c));
  if (needs_tuning(c)) ST(autotune(c));
  int32_t done = 0, conv = 0;
  const bool use_graph = !(c->cfg.flags & IVF_FLAG_NO_GRAPH);
  for (int32_t r = 1; r <= max_iter; ++r) {
    if (needs_tuning(c)) ST(autotune(c));
    const int target = c->alatest < 0 ? 0 : (c->alatest ^ 1);
    const int prev = c->alatest;
    if (use_graph && prev >= 0) {
      cudaGraphExec_t& g = c->graph[c->mcur][prev];
      long long& gk = c->graph_kernels[c->mcur][prev];
      if (!g) {
        cudaGraph_t graph = nullptr;
        const long long before = g_launches.load();
        CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        ivf_status s = enqueue_iteration(c, target, prev);
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        gk = g_launches.load() - before;
        g_launches.fetch_sub(gk);  // counted when the graph runs
        if (s != IVF_OK) {
          if (graph) cudaGraphDestroy(graph);
          return s;
        }
        if (e != cudaSuccess) return fail_cuda(c, "cudaStreamEndCapture", e);
        e = cudaGraphInstantiate(&g, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          g = nullptr;
          return fail_cuda(c, "cudaGraphInstantiate", e);
        }
      }
      CK(c, cudaGraphLaunch(g, c->stream));
      g_launches.fetch_add(gk);
    } else {
      ST(enqueue_iteration(c, target, prev));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->hc->status & STS_CAPACITY) {
      ST(redo_update_if_overflow(c, target));
      CK(c, cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
    }
    c->alatest = target;
    c->mcur ^= 1;
    c->iteration += 1;
    c->members_valid = true;
    c->e_cur = c->hc->ivf_e;
    ++done;
    ST(grow_head_if_needed(c, c->hc->heads_wanted));
    if (c->hc->status) ST(check_status(c));
    if (last_stats) fill_stats(c, last_stats);
    if (r >= 2 && c->hc->cnt[0] == 0) {
      conv = 1;
      break;
    }
  }
  if (iters_done) *iters_done = done;
  if (converged) *converged = conv;
  return IVF_OK;
}

ivf_status ivf_get_assign(ivf_ctx* c, int32_t* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  if (c->alatest < 0) return fail(c, IVF_E_STATE, "no assignment yet");
  CK(c, cudaMemcpyAsync(out, c->assign[c->alatest], sizeof(int32_t) * c->N, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return IVF_OK;
}

ivf_status ivf_get_best(ivf_ctx* c, float* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  if (c->alatest < 0) return fail(c, IVF_E_STATE, "no assignment yet");
  CK(c, cudaMemcpyAsync(out, c->best, sizeof(float) * c->N, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return IVF_OK;
}

ivf_status ivf_get_gap(ivf_ctx* c, float* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  if (c->alatest < 0) return fail(c, IVF_E_STATE, "no assignment yet");
  CK(c, cudaMemcpyAsync(out, c->gap, sizeof(float) * c->N, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return IVF_OK;
}

ivf_status ivf_get_err_bound(ivf_ctx* c, float* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  if (c->alatest < 0) return fail(c, IVF_E_STATE, "no assignment yet");
  CK(c, cudaMemcpyAsync(out, c->errb, sizeof(float) * c->N, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return IVF_OK;
}

ivf_status ivf_get_info(ivf_ctx* c, ivf_info* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  int64_t e = 0;
  if (c->means_set) {
    CK(c, cudaMemcpyAsync(&e, c->mptr[c->mcur] + c->Kt, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  out->n_docs = c->N;
  out->n_terms = c->Dt;
  out->nnz = c->nnz;
  out->k = (int32_t)c->Kt;
  out->n_instances = c->n_inst;
  out->ivf_entries = e;
  out->ivf_capacity = c->cap;
  out->k_tile = c->shape.k_tile;
  out->warps_per_block = c->shape.warps;
  out->iteration = c->iteration;
  out->storage = c->cfg.storage;
  out->device_bytes = c->bytes;
  out->dense_head_r = c->shape.head_r;
  out->dense_head_sub = c->shape.head_sub;
  out->dense_head_tensor = c->shape.tc ? 1 : 0;
  out->dense_head_theta = c->shape.head_theta;
  long long heads = 0;
  if (c->shape.head_r > 0) {
    CK(c, cudaMemcpy(&heads, &c->dc->heads, sizeof(long long), cudaMemcpyDeviceToHost));
  }
  out->dense_head_rows = heads;
  out->tile_major = c->shape.tmajor ? 1 : 0;
  return IVF_OK;
}

ivf_status ivf_get_means(ivf_ctx* c, int64_t* ptr, int32_t* term, double* val) {
  if (!c) return IVF_E_INVALID;
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  const int mb = c->mcur;
  std::vector<int64_t> hp(c->Kt + 1);
  CK(c, cudaMemcpyAsync(hp.data(), c->mptr[mb], sizeof(int64_t) * (c->Kt + 1), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const int64_t e = hp[c->Kt];
  if (ptr) CK(c, cudaMemcpy(ptr, hp.data(), sizeof(int64_t) * (c->Kt + 1), cudaMemcpyDefault));
  if (term) {
    std::vector<int32_t> ht(e);
    CK(c, cudaMemcpy(ht.data(), c->mterm[mb], sizeof(int32_t) * e, cudaMemcpyDeviceToHost));
    if (c->n_inst > 1) {
      for (int64_t j = 0; j < c->Kt; ++j) {
        int b = (int)(std::upper_bound(c->h_inst_clu.begin(), c->h_inst_clu.end(), (int32_t)j) - c->h_inst_clu.begin()) - 1;
        for (int64_t q = hp[j]; q < hp[j + 1]; ++q) ht[q] -= (int32_t)c->h_inst_toff[b];
      }
    }
    CK(c, cudaMemcpy(term, ht.data(), sizeof(int32_t) * e, cudaMemcpyDefault));
  }
  if (val) CK(c, cudaMemcpy(val, c->mval[mb], sizeof(double) * e, cudaMemcpyDefault));
  return IVF_OK;
}

ivf_status ivf_get_inverted_file(ivf_ctx* c, int64_t* term_ptr, int32_t* cid, float* w) {
  if (!c) return IVF_E_INVALID;
  if (!c->means_set) return fail(c, IVF_E_STATE, "means not set");
  CK(c, cudaStreamSynchronize(c->stream));
  int64_t e = 0;
  CK(c, cudaMemcpy(&e, c->term_ptr + c->Dt, sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (term_ptr) CK(c, cudaMemcpy(term_ptr, c->term_ptr, sizeof(int64_t) * (c->Dt + 1), cudaMemcpyDefault));
  if (cid) CK(c, cudaMemcpy(cid, c->cid32, sizeof(int32_t) * e, cudaMemcpyDefault));
  if (w) {
    std::vector<float> hw(e);
    if (c->cfg.storage == IVF_F32) {
      CK(c, cudaMemcpy(hw.data(), c->w, sizeof(float) * e, cudaMemcpyDeviceToHost));
    } else {
      std::vector<uint16_t> raw(e);
      CK(c, cudaMemcpy(raw.data(), c->w, sizeof(uint16_t) * e, cudaMemcpyDeviceToHost));
      for (int64_t q = 0; q < e; ++q) {
        if (c->cfg.storage == IVF_F16) {
          __half_raw hr;
          hr.x = raw[q];
          hw[q] = __half2float(__half(hr));
        } else {
          uint32_t bits = (uint32_t)raw[q] << 16;
          float f;
          memcpy(&f, &bits, 4);
          hw[q] = f;
        }
      }
    }
    CK(c, cudaMemcpy(w, hw.data(), sizeof(float) * e, cudaMemcpyDefault));
  }
  return IVF_OK;
}

ivf_status ivf_get_members(ivf_ctx* c, int64_t* cl_ptr, int32_t* members) {
  if (!c) return IVF_E_INVALID;
  if (!c->members_valid) return fail(c, IVF_E_STATE, "no update has run since the last change");
  CK(c, cudaStreamSynchronize(c->stream));
  if (cl_ptr) CK(c, cudaMemcpy(cl_ptr, c->cl_ptr, sizeof(int64_t) * (c->Kt + 1), cudaMemcpyDefault));
  if (members) {
    if (c->n_inst == 1) {
      CK(c, cudaMemcpy(members, c->members, sizeof(int32_t) * c->N, cudaMemcpyDefault));
    } else {
      std::vector<int32_t> hm(c->N);
      std::vector<int64_t> hcl(c->Kt + 1);
      CK(c, cudaMemcpy(hm.data(), c->members, sizeof(int32_t) * c->N, cudaMemcpyDeviceToHost));
      CK(c, cudaMemcpy(hcl.data(), c->cl_ptr, sizeof(int64_t) * (c->Kt + 1), cudaMemcpyDeviceToHost));
      for (int b = 0; b < c->n_inst; ++b)
        for (int64_t q = hcl[c->h_inst_clu[b]]; q < hcl[c->h_inst_clu[b + 1]]; ++q)
          hm[q] -= (int32_t)c->h_inst_docs[b];
      CK(c, cudaMemcpy(members, hm.data(), sizeof(int32_t) * c->N, cudaMemcpyDefault));
    }
  }
  return IVF_OK;
}

ivf_status ivf_set_assign(ivf_ctx* c, const int32_t* assign) {
  if (!c || !assign) return fail(c, IVF_E_INVALID, "null argument");
  std::vector<int32_t> h(c->N);
  CK(c, cudaMemcpy(h.data(), assign, sizeof(int32_t) * c->N, cudaMemcpyDefault));
  for (int b = 0; b < c->n_inst; ++b) {
    const int32_t kb = c->h_inst_clu[b + 1] - c->h_inst_clu[b];
    for (int64_t i = c->h_inst_docs[b]; i < c->h_inst_docs[b + 1]; ++i)
      if (h[i] < 0 || h[i] >= kb) return fail(c, IVF_E_INVALID, "assignment out of range");
  }
  const int target = c->alatest < 0 ? 0 : c->alatest;
  CK(c, cudaMemcpyAsync(c->assign[target], h.data(), sizeof(int32_t) * c->N, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->alatest = target;
  return IVF_OK;
}

ivf_status ivf_timing_reset(ivf_ctx* c, int32_t enable) {
  if (!c) return IVF_E_INVALID;
  CK(c, cudaStreamSynchronize(c->stream));
  c->tev_used = 0;
  c->tcalls.clear();
  c->timing = enable != 0;
  CK(c, cudaMemsetAsync(&c->dc->acc_entries, 0, 2 * sizeof(unsigned long long), c->stream));
  return IVF_OK;
}

ivf_status ivf_get_timing(ivf_ctx* c, ivf_timing* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  ST(read_counters(c));
  memset(out, 0, sizeof(*out));
  for (const auto& tc : c->tcalls) {
    float ms = 0.f;
    if (tc.kind == 0) {
      CK(c, cudaEventElapsedTime(&ms, c->tev[tc.e0], c->tev[tc.e0 + 1]));
      out->assign_kernel_ms += ms;
      CK(c, cudaEventElapsedTime(&ms, c->tev[tc.e0], c->tev[tc.e0 + 2]));
      out->assign_step_ms += ms;
      out->n_assign += 1;
    } else {
      CK(c, cudaEventElapsedTime(&ms, c->tev[tc.e0], c->tev[tc.e0 + 1]));
      out->update_ms += ms;
      out->n_update += 1;
    }
  }
  out->entries_visited = (int64_t)c->hc->acc_entries;
  out->n_rescored = (int64_t)c->hc->acc_rescored;
  return IVF_OK;
}

ivf_status ivfb_get_changed(ivf_ctx* c, int64_t* out) {
  if (!c || !out) return fail(c, IVF_E_INVALID, "null argument");
  CK(c, cudaMemcpyAsync(out, c->inst_changed, sizeof(int64_t) * c->n_inst, cudaMemcpyDefault, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return IVF_OK;
}

}  // extern "C"
