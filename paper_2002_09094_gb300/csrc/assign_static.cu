// ivf_assign_static: the assignment step without any device allocation.
//
// Some callers cannot allocate device memory at the point where they run
// the assignment: applications whose device memory is owned by their own pool
// or framework allocator, latency-critical loops that must not pay for (or
// synchronise the device on) a cudaMalloc after start-up, and embedded
// services that reserve all memory once.  They hold the objects, the inverted
// file, the FP64 means and the outputs in their own buffers; the only other
// memory the step needs -- work counters, object norms, and the queue of
// near-tie objects for the FP64 re-score -- lives here, in one file-scope
// static device array of fixed size.  Every GPU that loads the library holds
// that array until the process exits.
//
// Host code may not use the array's name as a device address: on the host it
// is only a stand-in symbol.  The device address comes from
// cudaGetSymbolAddress, looked up once per device (with that device current)
// on the first call there.
#include <mutex>

#include "../../include/ivf.h"
#include "common.cuh"
#include "kernels.cuh"

namespace {

using namespace ivfk;

// Layout of the scratch array (bytes).
constexpr size_t kCounters = 0;                                        // work, entries, rescored, flagged, status
constexpr size_t kTables = 32;                                         // instance tables of a single problem
constexpr size_t kNorms = 256;                                         // float[MAX_DOCS]
constexpr size_t kFlagObj = kNorms + 4ull * IVF_STATIC_MAX_DOCS;       // int32[MAX_DOCS]
constexpr size_t kFlagCnt = kFlagObj + 4ull * IVF_STATIC_MAX_DOCS;     // int32[MAX_DOCS]
constexpr size_t kBest = kFlagCnt + 4ull * IVF_STATIC_MAX_DOCS;        // float[MAX_DOCS] when best_out is NULL
constexpr size_t kGap = kBest + 4ull * IVF_STATIC_MAX_DOCS;            // float[MAX_DOCS] when gap_out is NULL
constexpr size_t kFlagCand = kGap + 4ull * IVF_STATIC_MAX_DOCS;        // int32[kCandInts]
constexpr size_t kCandInts = 32ull * IVF_STATIC_MAX_DOCS;               // candidate lists of kCandSlots objects
constexpr int64_t kCandSlots = (int64_t)(kCandInts / CAND_MAX);        // later flagged objects: all clusters
constexpr size_t kScratchBytes = kFlagCand + 4ull * kCandInts;
static_assert(kScratchBytes == IVF_STATIC_SCRATCH_BYTES, "scratch size stated in ivf.h");

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct Counters {
  unsigned long long work;
  unsigned long long entries;
  unsigned long long n_rescored;
  unsigned int n_flagged;
  unsigned int status;
};

struct Tables {
  int64_t docs[2];
  int64_t toff[2];
  int32_t clu[2];
  int32_t terms[1];
};

// Zero what must start at zero and write the single-instance tables.
__global__ void k_static_setup(unsigned char* scratch, int64_t n_docs, int32_t k, int32_t n_terms) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Counters* c = reinterpret_cast<Counters*>(scratch + kCounters);
  c->work = 0;
  c->entries = 0;
  c->n_rescored = 0;
  c->n_flagged = 0;
  c->status = 0;
  Tables* t = reinterpret_cast<Tables*>(scratch + kTables);
  t->docs[0] = 0;
  t->docs[1] = n_docs;
  t->toff[0] = 0;
  t->toff[1] = n_terms;
  t->clu[0] = 0;
  t->clu[1] = k;
  t->terms[0] = n_terms;
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_scratch[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Once per device, with that device current: the scratch array's device
// address and the kernel's shared-memory limit.
cudaError_t setup_device(int dev, unsigned char** scratch, int* sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = assign_prepare_i32ids(227 * 1024 / (int)sizeof(float) - 2 * CAND_MAX, 1);
    if (e != cudaSuccess) return e;
    g_dev_scratch[dev] = static_cast<unsigned char*>(p);
    g_num_sms[dev] = n;
  }
  *scratch = g_dev_scratch[dev];
  *sms = g_num_sms[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ivf_status ivf_assign_static(int64_t n_docs, const int64_t* row_ptr, const int32_t* term,
                                        const float* val, int64_t n_terms, int32_t k, const int64_t* term_ptr,
                                        const int32_t* cid, const float* w, const int64_t* mean_ptr,
                                        const int32_t* mean_term, const double* mean_val, int32_t* assign_out,
                                        float* best_out, float* gap_out, void* cuda_stream) {
  if (n_docs < 1 || n_docs > IVF_STATIC_MAX_DOCS || k < 1 || k > IVF_STATIC_MAX_K || (int64_t)k > n_docs ||
      n_terms < 1 || n_terms >= (int64_t(1) << 31))
    return IVF_E_INVALID;
  if (!row_ptr || !term || !val || !term_ptr || !cid || !w || !mean_ptr || !mean_term || !mean_val || !assign_out)
    return IVF_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IVF_E_CUDA;
  unsigned char* scratch = nullptr;
  int sms = 0;
  if (setup_device(dev, &scratch, &sms) != cudaSuccess) return IVF_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  const int tile_cap = (k + 3) & ~3;
  const size_t per_warp = ((size_t)tile_cap + 2 * CAND_MAX) * sizeof(float);
  int warps = (int)((227 * 1024) / per_warp);
  if (warps > 8) warps = 8;
  const int bps = assign_max_blocks_per_sm_i32ids(tile_cap, warps);
  if (bps < 1) return IVF_E_CUDA;

  Counters* ctr = reinterpret_cast<Counters*>(scratch + kCounters);
  Tables* tab = reinterpret_cast<Tables*>(scratch + kTables);
  float* nx = reinterpret_cast<float*>(scratch + kNorms);
  int32_t* flag_obj = reinterpret_cast<int32_t*>(scratch + kFlagObj);
  int32_t* flag_cnt = reinterpret_cast<int32_t*>(scratch + kFlagCnt);
  int32_t* flag_cand = reinterpret_cast<int32_t*>(scratch + kFlagCand);
  float* best = best_out ? best_out : reinterpret_cast<float*>(scratch + kBest);
  float* gap = gap_out ? gap_out : reinterpret_cast<float*>(scratch + kGap);

  k_static_setup<<<1, 32, 0, s>>>(scratch, n_docs, k, (int32_t)n_terms);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return IVF_E_CUDA;
  // the sign flag is not read here: the call uses the bound valid for signed values
  unsigned* negative = reinterpret_cast<unsigned*>(scratch + kTables + 128);
  // the caller's rows are read only (no term rebase: one instance, offset 0)
  if (launch_prepare_objects(n_docs, 0, 0, row_ptr, term, nullptr, val, nullptr, ST_F32, nx, 1,
                             tab->docs, tab->toff, tab->terms, 0, &ctr->status, negative, s) != cudaSuccess)
    return IVF_E_CUDA;

  AssignArgs a{};
  a.n_docs = n_docs;
  a.row_ptr = row_ptr;
  a.term = term;
  a.val = val;
  a.nx = nx;
  a.n_inst = 1;
  a.inst_docs = tab->docs;
  a.inst_clu = tab->clu;
  a.term_ptr = term_ptr;
  a.cid = cid;
  a.w = w;
  a.toff = nullptr;
  a.n_tiles_max = 0;
  a.k_tile = k;
  a.tiled = 0;
  a.tile_cap = tile_cap;
  a.storage = ST_F32;
  a.rescore = 1;
  a.assign = assign_out;
  a.best = best;
  a.gap = gap;
  a.work = &ctr->work;
  a.entries = &ctr->entries;
  a.n_flagged = &ctr->n_flagged;
  a.flag_obj = flag_obj;
  a.flag_cnt = flag_cnt;
  a.flag_cand = flag_cand;
  a.cand_slots = kCandSlots;
  a.nonneg = 0;
  if (launch_assign_i32ids(a, warps, bps * sms, s) != cudaSuccess) return IVF_E_CUDA;

  RescoreArgs r{};
  r.row_ptr = row_ptr;
  r.term = term;
  r.val32 = val;
  r.n_inst = 1;
  r.inst_docs = tab->docs;
  r.inst_clu = tab->clu;
  r.mptr = mean_ptr;
  r.mterm = mean_term;
  r.mval = mean_val;
  r.n_flagged = &ctr->n_flagged;
  r.flag_obj = flag_obj;
  r.flag_cnt = flag_cnt;
  r.flag_cand = flag_cand;
  r.assign = assign_out;
  r.best = best;
  r.gap = gap;
  r.n_rescored = &ctr->n_rescored;
  if (launch_rescore(r, 2 * sms, s) != cudaSuccess) return IVF_E_CUDA;
  return IVF_OK;
}
