// Update step of Algorithm 3 (IVF) on sm_103a, plus the inverted-file build
// shared with the initial means.
//
// The paper's update fills a dense w in R^D per cluster, divides by |C_j|,
// and appends (j, w_p / ||w||) to posting list p for every w_p != 0, visiting
// clusters in ascending j.  Here the same result is produced without a dense
// K x D array:
//   A5 group objects by cluster: stable radix sort of (cluster, object);
//   A6 member sums: every (term, value) of object i gets the key
//      (cluster(i), term); a stable LSD radix sort brings equal keys together
//      in ascending object id, and each run is summed sequentially in FP64
//      (the same order in which the oracle's dense accumulation adds them);
//   A7 normalise: ||s_j||^2 by a block per cluster in a fixed order (strided
//      partial sums by fused multiply-add, then a fixed tree), zero sums
//      dropped (w_p != 0), row offsets by a scan
//      over the clusters, rows written by a thread per run sum (by a block
//      per cluster for the rare clusters with an exactly zero sum);
//      empty clusters keep their previous mean or become empty;
//   A8 inverted file: a stable radix sort by term of the cluster-major means
//      gives posting lists in ascending cluster id; term_ptr by binary search.
// Dividing by |C_j| before normalising only rescales, so it is skipped.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "radix.cuh"

namespace ivfk {

namespace {

constexpr int T256 = 256;

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t g = ceil_div(n < 1 ? 1 : n, threads);
  if (g > cap) g = cap;
  return (unsigned)g;
}

template <typename T>
__device__ __forceinline__ int find_inst(const T* offs, int n_inst, T x) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename K>
__device__ __forceinline__ int64_t lower_bound_dev(const K* a, int64_t n, K x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------- A5 members

__global__ void k_member_keys(UpdateArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_docs; i += stride) {
    const int b = a.n_inst > 1 ? find_inst<int64_t>(a.inst_docs, a.n_inst, i) : 0;
    a.v32a[i] = (uint32_t)i;
    reinterpret_cast<uint32_t*>(a.k64a)[i] = (uint32_t)(a.inst_clu[b] + a.assign[i]);
  }
}

__global__ void k_member_out(UpdateArgs a, const uint32_t* keys, const uint32_t* vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_docs; i += stride)
    a.members[i] = (int32_t)vals[i];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= a.kt; j += stride)
    a.cl_ptr[j] = lower_bound_dev<uint32_t>(keys, a.n_docs, (uint32_t)j);
}

// ---------------------------------------- the objects' tuples by term (zeta)

// Warp per object: key = term, payload = (object << 32 | value bits).
__global__ void k_zeta_keys(const ZetaArgs z, uint32_t* keys, uint64_t* vals) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < z.n_docs; i += nw)
    for (int64_t h = z.row_ptr[i] + lane; h < z.row_ptr[i + 1]; h += 32) {
      keys[h] = (uint32_t)z.term[h];
      vals[h] = ((uint64_t)i << 32) | (uint64_t)__float_as_uint(z.val32[h]);
    }
}

__global__ void k_zeta_ptr(const ZetaArgs z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= z.dt; s += stride)
    z.zptr[s] = lower_bound_dev<uint32_t>(z.zterm, z.nnz, (uint32_t)s);
}

// ------------------------------------------------------- A6 member sums

// Key = global cluster of the tuple's object, payload = (term << 32 | value
// bits).  A stable sort on this key alone orders the tuples by (cluster,
// term, object): zeta is already in (term, object) order.
__global__ void k_zc_keys(UpdateArgs a, uint32_t* keys, uint64_t* vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.nnz; q += stride) {
    const uint64_t ov = a.zov[q];
    const int64_t o = (int64_t)(ov >> 32);
    const int b = a.n_inst > 1 ? find_inst<int64_t>(a.inst_docs, a.n_inst, o) : 0;
    keys[q] = (uint32_t)(a.inst_clu[b] + a.assign[o]);
    vals[q] = ((uint64_t)a.zterm[q] << 32) | (ov & 0xFFFFFFFFull);
  }
}

// Run heads of (cluster, term) in that order: flags[e] = 1 on the first
// entry of a run (heads_to_starts turns them into the run starts).
__global__ void k_zc_heads(const uint32_t* cl, const uint64_t* tv, const int64_t* d_n, uint32_t* flags) {
  const int64_t n = *d_n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
    flags[e] = (e == 0 || cl[e] != cl[e - 1] || (tv[e] >> 32) != (tv[e - 1] >> 32)) ? 1u : 0u;
}

__global__ void k_starts(const uint32_t* scanned, const int64_t* d_n, uint32_t* starts, int64_t* d_u) {
  const int64_t n = *d_n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
    if (scanned[e + 1] != scanned[e]) starts[scanned[e]] = (uint32_t)e;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    starts[scanned[n]] = (uint32_t)n;
    *d_u = (int64_t)scanned[n];
  }
}

// Each run of one (cluster, term) summed in FP64 in its (ascending object)
// order; key (cluster, the term's id inside its instance: a cluster's terms
// all come from its instance).
__global__ void k_zc_segsum(const UpdateArgs a, const uint32_t* cl, const uint64_t* tv) {
  const int64_t u_n = *a.d_u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < u_n; u += stride) {
    const uint32_t s0 = a.starts[u], s1 = a.starts[u + 1];
    // sequential from the first value (0 + v would be v, so that add is skipped)
    double s = (double)__uint_as_float((uint32_t)tv[s0]);
    for (uint32_t e = s0 + 1; e < s1; ++e) s = __dadd_rn(s, (double)__uint_as_float((uint32_t)tv[e]));
    const uint32_t gc = cl[s0];
    const int32_t t0 = a.n_inst > 1 ? (int32_t)a.inst_toff[find_inst<int32_t>(a.inst_clu, a.n_inst, (int32_t)gc)] : 0;
    a.ukey[u] = ((uint64_t)gc << a.tbits) | (uint64_t)(uint32_t)((int32_t)(tv[s0] >> 32) - t0);
    a.usum[u] = s;
  }
}

// ------------------------------------------------------------ A7 normalise

__global__ void k_uptr(UpdateArgs a) {
  const int64_t u_n = *a.d_u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= a.kt; j += stride)
    a.uptr[j] = lower_bound_dev<uint64_t>(a.ukey, u_n, (uint64_t)j << a.tbits);
}

// Block per cluster: ||s_j||^2, the count of nonzero elements and the
// length of the new mean row.  Thread t sums the squares of elements
// u0 + t, u0 + t + 256, ... in order; the 32 lanes of a warp are combined by
// a fixed butterfly and the 8 warp totals in warp order.  The order depends
// only on the cluster's element range, never on the launch shape, so the
// result is bit-reproducible; long rows take E_j / 256 dependent steps.
constexpr int kNormThreads = 256;
__global__ void __launch_bounds__(kNormThreads) k_cluster_norm(UpdateArgs a) {
  __shared__ double wsum[kNormThreads / 32];
  __shared__ int wnz[kNormThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t j = blockIdx.x; j < a.kt; j += gridDim.x) {
    const int64_t u0 = a.uptr[j], u1 = a.uptr[j + 1];
    double n2 = 0.0;
    int nz = 0;
    for (int64_t u = u0 + threadIdx.x; u < u1; u += kNormThreads) {
      const double v = a.usum[u];
      n2 = __fma_rn(v, v, n2);
      nz += (v != 0.0) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n2 = __dadd_rn(n2, __shfl_xor_sync(IVF_FULL_MASK, n2, o));
      nz += __shfl_xor_sync(IVF_FULL_MASK, nz, o);
    }
    if (lane == 0) {
      wsum[warp] = n2;
      wnz[warp] = nz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      int64_t cnt = 0;
      for (int w = 0; w < kNormThreads / 32; ++w) {
        t = __dadd_rn(t, wsum[w]);
        cnt += wnz[w];
      }
      const double nrm = __dsqrt_rn(t);
      a.sum_norm[j] = nrm;
      a.rnorm[j] = nrm > 0.0 ? __drcp_rn(nrm) : 0.0;
      a.zrun[j] = cnt != u1 - u0 ? 1 : 0;
      int64_t len;
      if (nrm > 0.0)
        len = cnt;
      else
        len = a.empty_policy == 0 ? (a.mptr_old[j + 1] - a.mptr_old[j]) : 0;
      a.newlen[j] = len;
    }
    __syncthreads();
  }
}

// s / ||s_j|| as s * y with y = RN(1 / ||s_j||): one FP64 multiply instead
// of a division (FP64 issues at a small fraction of the FP32 rate on this
// part: a division per run sum took 1.4 ms at 4.8e7 sums, a multiply plus a
// Markstein correction 0.9 ms).  Within two ulps of the quotient.
__device__ __forceinline__ double div_by_norm(double s, double y) { return __dmul_rn(s, y); }

// Thread per run sum u of a cluster j with ||s_j|| > 0 and no zero run sum:
// mu_j element = s / ||s_j|| at mptr_new[j] + (u - uptr[j]) (every run is
// kept, so a run's rank is its offset).  Over the whole grid, so the largest
// clusters (hundreds of thousands of runs) leave no tail.
__global__ void k_write_flat(UpdateArgs a) {
  if (a.mptr_new[a.kt] > a.cap) return;  // k_write_rows raises STS_CAPACITY
  const uint64_t tmask = (a.tbits >= 64) ? ~0ull : ((1ull << a.tbits) - 1ull);
  const int64_t u_n = *a.d_u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool neg = false;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < u_n; u += stride) {
    const uint64_t key = a.ukey[u];
    const int32_t j = (int32_t)(key >> a.tbits);
    const double nrm = a.sum_norm[j];
    if (!(nrm > 0.0) || a.zrun[j] != 0) continue;
    const int32_t t0 = a.n_inst > 1 ? (int32_t)a.inst_toff[find_inst<int32_t>(a.inst_clu, a.n_inst, j)] : 0;
    const double s = a.usum[u];
    const int64_t p = a.mptr_new[j] + (u - a.uptr[j]);
    a.mterm_new[p] = (int32_t)(key & tmask) + t0;
    a.mval_new[p] = div_by_norm(s, a.rnorm[j]);
    a.mclu_new[p] = j;
    neg |= s < 0.0;
  }
  if (__any_sync(IVF_FULL_MASK, neg) && (threadIdx.x & 31) == 0) atomicOr(a.means_negative, 1u);
}

// Block per cluster with ||s_j|| > 0 and at least one zero run sum (exact
// cancellation, signed data only): its mean row, mu_j element = s / ||s_j||
// for every nonzero run sum in term order, written at mptr_new[j] + (the
// sum's rank among the cluster's nonzero sums: a block-wide running count,
// 256 sums at a time).  Clusters with ||s_j|| = 0 are left to k_copy_kept,
// the rest to k_write_flat.
__global__ void __launch_bounds__(kNormThreads) k_write_rows(UpdateArgs a) {
  __shared__ int wcount[kNormThreads / 32];
  if (a.mptr_new[a.kt] > a.cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, (unsigned)STS_CAPACITY);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t tmask = (a.tbits >= 64) ? ~0ull : ((1ull << a.tbits) - 1ull);
  bool neg = false;
  for (int64_t j = blockIdx.x; j < a.kt; j += gridDim.x) {
    const double nrm = a.sum_norm[j];
    if (!(nrm > 0.0) || a.zrun[j] == 0) continue;  // uniform over the block
    const double y = a.rnorm[j];
    const int32_t t0 = a.n_inst > 1 ? (int32_t)a.inst_toff[find_inst<int32_t>(a.inst_clu, a.n_inst, (int32_t)j)] : 0;
    const int64_t u0 = a.uptr[j], u1 = a.uptr[j + 1];
    int64_t o = a.mptr_new[j];
    for (int64_t c0 = u0; c0 < u1; c0 += kNormThreads) {
      const int64_t u = c0 + threadIdx.x;
      const double s = u < u1 ? a.usum[u] : 0.0;
      const bool keep = s != 0.0;
      const unsigned m = __ballot_sync(IVF_FULL_MASK, keep);
      if (lane == 0) wcount[warp] = __popc(m);
      __syncthreads();
      int before = 0, total = 0;
      for (int w = 0; w < kNormThreads / 32; ++w) {
        before += w < warp ? wcount[w] : 0;
        total += wcount[w];
      }
      if (keep) {
        const int64_t p = o + before + __popc(m & ((1u << lane) - 1u));
        a.mterm_new[p] = (int32_t)(a.ukey[u] & tmask) + t0;
        a.mval_new[p] = div_by_norm(s, y);
        a.mclu_new[p] = (int32_t)j;
        neg |= s < 0.0;
      }
      o += total;
      __syncthreads();
    }
  }
  if (__any_sync(IVF_FULL_MASK, neg) && lane == 0) atomicOr(a.means_negative, 1u);
}

// Warp per cluster with no members (or a zero sum) under empty_policy 0:
// copy the previous row.
__global__ void k_copy_kept(UpdateArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (a.empty_policy != 0 || a.mptr_new[a.kt] > a.cap) return;
  bool neg = false;
  for (int64_t j = gw; j < a.kt; j += nw) {
    if (a.sum_norm[j] > 0.0) continue;
    const int64_t dst = a.mptr_new[j];
    const int64_t o0 = a.mptr_old[j], o1 = a.mptr_old[j + 1];
    for (int64_t q = lane; q < o1 - o0; q += 32) {
      a.mterm_new[dst + q] = a.mterm_old[o0 + q];
      const double v = a.mval_old[o0 + q];
      a.mval_new[dst + q] = v;
      a.mclu_new[dst + q] = (int32_t)j;
      neg |= !(v >= 0.0);
    }
  }
  if (__any_sync(IVF_FULL_MASK, neg) && lane == 0) atomicOr(a.means_negative, 1u);
}

// ------------------------------------------------------- A8 inverted file

// Key = term; payload = (local cluster << 32 | the value in the storage
// type's bits), carried through the sort so the fill reads it in order.
template <typename WT>
__global__ void k_ivf_keys(IvfBuildArgs a) {
  const int64_t e_n = a.mptr[a.kt];
  const int64_t n = e_n > a.cap ? 0 : e_n;
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.d_e = n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int32_t gc = a.mclu[e];
    const int b = a.n_inst > 1 ? find_inst<int32_t>(a.inst_clu, a.n_inst, (int32_t)gc) : 0;
    const uint32_t local = (uint32_t)(gc - a.inst_clu[b]);
    const WT w = from_f64<WT>(a.mval[e]);
    uint32_t bits;
    if constexpr (sizeof(WT) == 4)
      bits = __float_as_uint(*reinterpret_cast<const float*>(&w));
    else
      bits = (uint32_t)(*reinterpret_cast<const uint16_t*>(&w));
    a.v32a[e] = (uint32_t)a.mterm[e];
    a.v64a[e] = ((uint64_t)local << 32) | bits;
  }
}

__global__ void k_term_ptr(IvfBuildArgs a, const uint32_t* sorted_terms) {
  const int64_t n = *a.d_e;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= a.dt; p += stride)
    a.term_ptr[p] = lower_bound_dev<uint32_t>(sorted_terms, n, (uint32_t)p);
}

template <typename WT>
__global__ void k_ivf_fill(IvfBuildArgs a, const uint64_t* cv) {
  const int64_t n = *a.d_e;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const uint64_t x = cv[q];
    const int32_t local = (int32_t)(x >> 32);
    a.cid32[q] = local;
    a.cid16[q] = (uint16_t)(local & 0xFFFF);
    if constexpr (sizeof(WT) == 4)
      static_cast<uint32_t*>(a.w)[q] = (uint32_t)x;
    else
      static_cast<uint16_t*>(a.w)[q] = (uint16_t)x;
  }
}

// Per (term, tile): offset inside the term's list of the first entry whose
// cluster id reaches tile * k_tile.
__global__ void k_toff(IvfBuildArgs a) {
  const int64_t per = (int64_t)a.n_tiles_max + 1;
  const int64_t total = a.dt * per;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
    const int64_t p = x / per;
    const int64_t tt = x - p * per;
    const int64_t tb = a.term_ptr[p], te = a.term_ptr[p + 1];
    const int64_t target = tt * (int64_t)a.k_tile;
    int64_t lo = tb, hi = te;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)a.cid32[mid] < target)
        lo = mid + 1;
      else
        hi = mid;
    }
    a.toff[x] = (int32_t)(lo - tb);
  }
}

// ------------------------------------------------ dense head rows (IFN form)

// A term whose posting list holds at least head_min_nc clusters is stored as
// a dense row of kpad values (zeros where the list has no entry): the
// paper's full inverted file (IFN) restricted to the densest lists.
__global__ void k_head_flags(IvfBuildArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.dt; p += stride) {
    int64_t min_nc = a.head_min_nc;
    if (a.n_inst > 1) {  // theta * K of the term's own instance
      const int b = find_inst<int64_t>(a.inst_toff, a.n_inst, p);
      const int64_t kb = a.inst_clu[b + 1] - a.inst_clu[b];
      min_nc = (int64_t)ceilf(a.head_theta * (float)kb);
      if (min_nc < 1) min_nc = 1;
    }
    a.hflags[p] = (a.term_ptr[p + 1] - a.term_ptr[p] >= min_nc) ? 1u : 0u;
  }
}

__global__ void k_head_slots(IvfBuildArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.dt; p += stride) {
    const uint32_t s = a.hflags[p];
    const bool head = a.hflags[p + 1] != s && (int64_t)s < a.head_max;
    a.head_slot[p] = head ? (int32_t)s : -1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t tot = (int64_t)a.hflags[a.dt];
    *a.d_heads = tot < a.head_max ? tot : a.head_max;
    if (a.d_heads_wanted) *a.d_heads_wanted = tot;
  }
}

template <typename WT>
__global__ void k_head_zero(IvfBuildArgs a) {
  WT* wd = static_cast<WT*>(a.wd);
  const int64_t n = (a.zero_rows > 0 ? a.zero_rows : *a.d_heads) * a.kpad;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) wd[x] = from_f32<WT>(0.f);
}

// Warp per term: copy a head term's list into its dense row.
template <typename WT>
__global__ void k_head_fill(IvfBuildArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  WT* wd = static_cast<WT*>(a.wd);
  const WT* w = static_cast<const WT*>(a.w);
  for (int64_t p = gw; p < a.dt; p += nw) {
    const int32_t s = a.head_slot[p];
    if (s < 0) continue;
    WT* row = wd + (int64_t)s * a.kpad;
    for (int64_t q = a.term_ptr[p] + lane; q < a.term_ptr[p + 1]; q += 32) row[a.cid32[q]] = w[q];
  }
}

// ------------------------------------------------------ means from rows

__global__ void k_normalise_rows(int64_t kt, const int64_t* mptr, double* mval, int32_t* mclu, int64_t dt,
                                 const int32_t* mterm, unsigned* status, int normalise, unsigned* negative) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < kt; j += stride) {
    const int64_t r0 = mptr[j], r1 = mptr[j + 1];
    double n2 = 0.0;
    bool ok = r1 >= r0;
    bool neg = false;
    for (int64_t e = r0; e < r1; ++e) {
      const double v = mval[e];
      neg |= !(v >= 0.0);
      n2 = __dadd_rn(n2, __dmul_rn(v, v));
      const int32_t t = mterm[e];
      if (t < 0 || (int64_t)t >= dt || (e > r0 && mterm[e - 1] >= t) || !isfinite(v)) ok = false;
    }
    if ((normalise && !(n2 > 0.0)) || !isfinite(n2) || !ok) {
      atomicOr(status, (unsigned)STS_BAD_MEANS);
      continue;
    }
    if (neg) atomicOr(negative, 1u);
    const double nrm = __dsqrt_rn(n2);
    for (int64_t e = r0; e < r1; ++e) {
      if (normalise) mval[e] = __ddiv_rn(mval[e], nrm);
      mclu[e] = (int32_t)j;
    }
  }
}

__global__ void k_gather_lens(int64_t kt, const int32_t* doc_ids, const int64_t* row_ptr, int64_t* lens) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < kt; j += stride) {
    const int64_t d = doc_ids[j];
    lens[j] = row_ptr[d + 1] - row_ptr[d];
  }
}

__global__ void k_gather_copy(int64_t kt, const int32_t* doc_ids, const int64_t* row_ptr, const int32_t* term,
                              const float* val32, const int64_t* mptr, int32_t* mterm, double* mval) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = gw; j < kt; j += nw) {
    const int64_t d = doc_ids[j];
    const int64_t r0 = row_ptr[d], len = row_ptr[d + 1] - r0, o = mptr[j];
    for (int64_t q = lane; q < len; q += 32) {
      mterm[o + q] = term[r0 + q];
      mval[o + q] = (double)val32[r0 + q];
    }
  }
}

// --------------------------------------------------------- objects

template <typename WT>
// term_rebase: the same array as term, written in place with global term ids
// when an instance's term offset is non-zero; null = never written (the
// caller's rows are read only).
__global__ void k_prepare_objects(int64_t n_docs, const int64_t* row_ptr, const int32_t* term,
                                  int32_t* term_rebase, const float* val32,
                                  WT* val_store, float* nx, int32_t n_inst, const int64_t* inst_docs,
                                  const int64_t* inst_toff, const int32_t* inst_terms, int validate,
                                  unsigned* status, unsigned* negative) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_docs; i += nw) {
    const int b = n_inst > 1 ? find_inst<int64_t>(inst_docs, n_inst, i) : 0;
    const int64_t toff = inst_toff[b];
    const int32_t d_local = inst_terms[b];
    const int64_t r0 = row_ptr[i], r1 = row_ptr[i + 1];
    double ss = 0.0;
    bool bad = r1 < r0;
    bool neg = false;
    for (int64_t h = r0 + lane; h < r1; h += 32) {
      const int32_t t = term[h];
      const float v = val32[h];
      neg |= !(v >= 0.f);
      if (validate) {
        if (t < 0 || t >= d_local || !isfinite(v)) bad = true;
        if (h > r0 && term[h - 1] >= t) bad = true;
      }
      const double dv = f32_bits_to_f64(__float_as_uint(v));
      ss = __fma_rn(dv, dv, ss);
      if (val_store) val_store[h] = from_f32<WT>(v);
    }
    __syncwarp();
    if (toff != 0 && term_rebase != nullptr)
      for (int64_t h = r0 + lane; h < r1; h += 32) term_rebase[h] = (int32_t)(term[h] + toff);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(IVF_FULL_MASK, ss, o);
    const bool any_bad = __any_sync(IVF_FULL_MASK, bad);
    const bool any_neg = __any_sync(IVF_FULL_MASK, neg);
    if (lane == 0) {
      // an upper bound on ||x_i||: the FP64 sum is within a few ulps, then round up
      nx[i] = __double2float_ru(__dsqrt_ru(ss * (1.0 + 1e-12)));
      if (any_bad) atomicOr(status, (unsigned)STS_BAD_ROWS);
      if (any_neg) atomicOr(negative, 1u);
    }
  }
}

// row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz; a violation sets STS_BAD_ROWS.
__global__ void k_check_row_ptr(const int64_t* rp, int64_t n, int64_t nnz, unsigned* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) bad |= rp[i + 1] < rp[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) bad |= rp[0] != 0 || rp[n] != nnz;
  if (bad) atomicOr(status, (unsigned)STS_BAD_ROWS);
}

}  // namespace

// A7 from the run sums of A6 (ukey, usum, *d_u <= u_max): norms, new row
// lengths, prefix sums, the normalised entries, kept rows of empty clusters.
cudaError_t launch_means_from_sums(const UpdateArgs& a, int64_t u_max, cudaStream_t s) {
  const unsigned gK = grid_for(a.kt + 1, T256, 8192);
  k_uptr<<<gK, T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  k_cluster_norm<<<(unsigned)std::min<int64_t>(a.kt, 16384), kNormThreads, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  IVF_CU(exclusive_scan_i64(a.newlen, a.mptr_new, a.kt, a.temp, s));
  k_write_flat<<<grid_for(u_max, T256, 16384), T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  k_write_rows<<<(unsigned)std::min<int64_t>(a.kt, 16384), kNormThreads, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  k_copy_kept<<<grid_for(a.kt * 32, T256, 8192), T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

// ------------------------------------------ member sums gathered from shards

__global__ void k_part_keys1(const PartialArgs p, uint32_t* keys, uint32_t* vals) {
  const int64_t n = *p.d_n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    keys[e] = (uint32_t)p.term[e];
    vals[e] = (uint32_t)e;
  }
}

__global__ void k_part_keys2(const PartialArgs p, const uint32_t* perm1, uint32_t* keys, uint32_t* vals) {
  const int64_t n = *p.d_n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const uint32_t q = perm1[e];
    keys[e] = (uint32_t)p.cluster[q];
    vals[e] = q;
  }
}

__global__ void k_part_heads(const PartialArgs p, const uint32_t* perm, uint32_t* flags) {
  const int64_t n = *p.d_n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    bool head = e == 0;
    if (!head) {
      const uint32_t q = perm[e], r = perm[e - 1];
      head = p.cluster[q] != p.cluster[r] || p.term[q] != p.term[r];
    }
    flags[e] = head ? 1u : 0u;
  }
}

// Run sums in the given (shard) order; key (cluster, term) as A6 makes it.
__global__ void k_part_segsum(const UpdateArgs a, const PartialArgs p, const uint32_t* perm) {
  const int64_t u_n = *a.d_u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < u_n; u += stride) {
    const uint32_t s0 = a.starts[u], s1 = a.starts[u + 1];
    double s = 0.0;
    for (uint32_t e = s0; e < s1; ++e) s = __dadd_rn(s, p.sum[perm[e]]);
    const uint32_t q = perm[s0];
    a.ukey[u] = ((uint64_t)(uint32_t)p.cluster[q] << a.tbits) | (uint64_t)(uint32_t)p.term[q];
    a.usum[u] = s;
  }
}

__global__ void k_part_out(const UpdateArgs a, int32_t* cluster, int32_t* term, double* sum) {
  const int64_t u_n = *a.d_u;
  const uint64_t tmask = (1ull << a.tbits) - 1ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < u_n; u += stride) {
    const uint64_t k = a.ukey[u];
    cluster[u] = (int32_t)(k >> a.tbits);
    term[u] = (int32_t)(k & tmask);
    sum[u] = a.usum[u];
  }
}

__global__ void k_check_partials(int64_t n, const int32_t* cluster, const int32_t* term, int32_t k, int32_t d,
                                 unsigned* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
    bad |= cluster[e] < 0 || cluster[e] >= k || term[e] < 0 || term[e] >= d;
  if (__any_sync(IVF_FULL_MASK, bad) && (threadIdx.x & 31) == 0) atomicOr(status, (unsigned)STS_BAD_ROWS);
}

cudaError_t launch_check_partials(int64_t n, const int32_t* cluster, const int32_t* term, int32_t k, int32_t d,
                                  unsigned* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_check_partials<<<grid_for(n, T256, 8192), T256, 0, s>>>(n, cluster, term, k, d, status);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_partial_out(const UpdateArgs& a, int64_t u_max, int32_t* cluster, int32_t* term, double* sum,
                               cudaStream_t s) {
  k_part_out<<<grid_for(u_max, T256, 16384), T256, 0, s>>>(a, cluster, term, sum);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_update_from_partials(const UpdateArgs& a, const PartialArgs& p, cudaStream_t s) {
  const unsigned gP = grid_for(p.n_max, T256, 16384);
  uint32_t* ka = reinterpret_cast<uint32_t*>(a.k64a);
  uint32_t* kb = reinterpret_cast<uint32_t*>(a.k64b);
  // stable by term, then stably by cluster: (cluster, term) order, equal keys in shard order
  k_part_keys1<<<gP, T256, 0, s>>>(p, ka, a.v32a);
  IVF_LAUNCH_CHECK();
  bool alt = false;
  IVF_CU(radix_sort_u32(ka, kb, a.v32a, a.v32b, p.d_n, p.n_max, a.tbits, a.temp, s, &alt));
  const uint32_t* perm1 = alt ? a.v32b : a.v32a;
  uint32_t* k2 = alt ? ka : kb;
  uint32_t* v2 = alt ? a.v32a : a.v32b;
  k_part_keys2<<<gP, T256, 0, s>>>(p, perm1, k2, v2);
  IVF_LAUNCH_CHECK();
  bool alt2 = false;
  uint32_t* k2b = alt ? kb : ka;
  uint32_t* v2b = alt ? a.v32b : a.v32a;
  IVF_CU(radix_sort_u32(k2, k2b, v2, v2b, p.d_n, p.n_max, a.kbits, a.temp, s, &alt2));
  const uint32_t* perm = alt2 ? v2b : v2;
  k_part_heads<<<gP, T256, 0, s>>>(p, perm, a.flags);
  IVF_LAUNCH_CHECK();
  IVF_CU(exclusive_scan_u32(a.flags, a.flags, p.n_max, a.temp, s));
  k_starts<<<gP, T256, 0, s>>>(a.flags, p.d_n, a.starts, a.d_u);
  IVF_LAUNCH_CHECK();
  k_part_segsum<<<gP, T256, 0, s>>>(a, p, perm);
  IVF_LAUNCH_CHECK();
  return launch_means_from_sums(a, p.n_max, s);
}

// A5 (members) and A6 (run sums per (cluster, term)).
cudaError_t launch_member_sums(const UpdateArgs& a, cudaStream_t s) {
  const unsigned gN = grid_for(a.n_docs, T256, 8192);
  // A5: C_j as a stable counting sort of objects by cluster
  k_member_keys<<<gN, T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  {
    uint32_t* ka = reinterpret_cast<uint32_t*>(a.k64a);
    uint32_t* kb = reinterpret_cast<uint32_t*>(a.k64b);
    bool alt = false;
    IVF_CU(radix_sort_u32(ka, kb, a.v32a, a.v32b, a.d_n, a.n_docs, a.kbits, a.temp, s, &alt));
    k_member_out<<<grid_for(a.n_docs > a.kt ? a.n_docs : a.kt + 1, T256, 8192), T256, 0, s>>>(
        a, alt ? kb : ka, alt ? a.v32b : a.v32a);
    IVF_LAUNCH_CHECK();
  }
  // A6: zeta's tuples stably sorted by cluster alone -- (cluster, term,
  // object) order -- then FP64 run sums per (cluster, term)
  const unsigned gE = grid_for(a.nnz, T256, 16384);
  k_zc_keys<<<gE, T256, 0, s>>>(a, a.v32a, a.k64a);
  IVF_LAUNCH_CHECK();
  bool alt = false;
  IVF_CU(radix_sort_u32_wide(a.v32a, a.v32b, a.k64a, a.k64b, a.d_nnz, a.nnz, a.kbits, a.temp, s, &alt));
  const uint32_t* cl = alt ? a.v32b : a.v32a;
  const uint64_t* tv = alt ? a.k64b : a.k64a;
  k_zc_heads<<<gE, T256, 0, s>>>(cl, tv, a.d_nnz, a.flags);
  IVF_LAUNCH_CHECK();
  IVF_CU(heads_to_starts(a.flags, a.nnz, a.starts, a.d_u, a.temp, s));
  k_zc_segsum<<<gE, T256, 0, s>>>(a, cl, tv);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_update_means(const UpdateArgs& a, cudaStream_t s) {
  IVF_CU(launch_member_sums(a, s));
  return launch_means_from_sums(a, a.nnz, s);  // A7
}

cudaError_t launch_build_zeta(const ZetaArgs& z, cudaStream_t s) {
  // a stable sort by term of (term, object|value); the passes ping-pong
  // between the scratch pair and zeta itself, started so the result lands in zeta
  const int passes = (z.tbits + 7) / 8;
  uint32_t* k0 = (passes & 1) ? z.k32 : z.zterm;
  uint32_t* k1 = (passes & 1) ? z.zterm : z.k32;
  uint64_t* v0 = (passes & 1) ? z.v64 : z.zov;
  uint64_t* v1 = (passes & 1) ? z.zov : z.v64;
  k_zeta_keys<<<grid_for(z.n_docs * 32, T256, 16384), T256, 0, s>>>(z, k0, v0);
  IVF_LAUNCH_CHECK();
  bool alt = false;
  IVF_CU(radix_sort_u32_wide(k0, k1, v0, v1, z.d_nnz, z.nnz, z.tbits, z.temp, s, &alt));
  k_zeta_ptr<<<grid_for(z.dt + 1, T256, 16384), T256, 0, s>>>(z);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_build_ivf(const IvfBuildArgs& a, cudaStream_t s) {
  const unsigned gE = grid_for(a.cap, T256, 16384);
  switch (a.storage) {
    case ST_F16:
      k_ivf_keys<__half><<<gE, T256, 0, s>>>(a);
      break;
    case ST_BF16:
      k_ivf_keys<__nv_bfloat16><<<gE, T256, 0, s>>>(a);
      break;
    default:
      k_ivf_keys<float><<<gE, T256, 0, s>>>(a);
      break;
  }
  IVF_LAUNCH_CHECK();
  bool alt = false;
  IVF_CU(radix_sort_u32_wide(a.v32a, a.v32b, a.v64a, a.v64b, a.d_e, a.cap, a.tbits, a.temp, s, &alt));
  const uint32_t* terms = alt ? a.v32b : a.v32a;
  const uint64_t* cv = alt ? a.v64b : a.v64a;
  k_term_ptr<<<grid_for(a.dt + 1, T256, 16384), T256, 0, s>>>(a, terms);
  IVF_LAUNCH_CHECK();
  switch (a.storage) {
    case ST_F16:
      k_ivf_fill<__half><<<gE, T256, 0, s>>>(a, cv);
      break;
    case ST_BF16:
      k_ivf_fill<__nv_bfloat16><<<gE, T256, 0, s>>>(a, cv);
      break;
    default:
      k_ivf_fill<float><<<gE, T256, 0, s>>>(a, cv);
      break;
  }
  IVF_LAUNCH_CHECK();
  if (a.toff) IVF_CU(launch_build_toff(a, s));
  if (a.head_slot) IVF_CU(launch_build_head(a, s));
  return cudaSuccess;
}

cudaError_t launch_build_head(const IvfBuildArgs& a, cudaStream_t s) {
  const unsigned gD = grid_for(a.dt, T256, 16384);
  k_head_flags<<<gD, T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  IVF_CU(exclusive_scan_u32(a.hflags, a.hflags, a.dt, a.temp, s));
  k_head_slots<<<gD, T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  const unsigned gW = grid_for((a.zero_rows > a.head_max ? a.zero_rows : a.head_max) * a.kpad, T256, 16384);
  const unsigned gF = grid_for(a.dt * 32, T256, 16384);
  switch (a.storage) {
    case ST_F16:
      k_head_zero<__half><<<gW, T256, 0, s>>>(a);
      IVF_LAUNCH_CHECK();
      k_head_fill<__half><<<gF, T256, 0, s>>>(a);
      break;
    case ST_BF16:
      k_head_zero<__nv_bfloat16><<<gW, T256, 0, s>>>(a);
      IVF_LAUNCH_CHECK();
      k_head_fill<__nv_bfloat16><<<gF, T256, 0, s>>>(a);
      break;
    default:
      k_head_zero<float><<<gW, T256, 0, s>>>(a);
      IVF_LAUNCH_CHECK();
      k_head_fill<float><<<gF, T256, 0, s>>>(a);
      break;
  }
  IVF_LAUNCH_CHECK();
  if (a.wdT != nullptr) IVF_CU(launch_transpose16(a.wd, a.head_max, a.kpad, a.wdT, a.ldt, s));
  return cudaSuccess;
}

cudaError_t launch_build_toff(const IvfBuildArgs& a, cudaStream_t s) {
  if (a.toff == nullptr || a.k_tile <= 0) return cudaErrorInvalidValue;
  k_toff<<<grid_for(a.dt * (a.n_tiles_max + 1), T256, 16384), T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_normalise_rows(int64_t kt, const int64_t* mptr, double* mval, int32_t* mclu, int64_t dt,
                                  const int32_t* mterm, unsigned* status, int normalise, unsigned* negative,
                                  cudaStream_t s) {
  k_normalise_rows<<<grid_for(kt, 64, 8192), 64, 0, s>>>(kt, mptr, mval, mclu, dt, mterm, status, normalise,
                                                         negative);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_gather_rows(int64_t kt, const int32_t* doc_ids, const int64_t* row_ptr, const int32_t* term,
                               const float* val32, int64_t* lens_then_ptr, int32_t* mterm, double* mval, void* temp,
                               cudaStream_t s, int phase) {
  if (phase == 0) {
    k_gather_lens<<<grid_for(kt, T256, 8192), T256, 0, s>>>(kt, doc_ids, row_ptr, lens_then_ptr);
    IVF_LAUNCH_CHECK();
    IVF_CU(exclusive_scan_i64(lens_then_ptr, lens_then_ptr, kt, temp, s));
  } else {
    k_gather_copy<<<grid_for(kt * 32, T256, 8192), T256, 0, s>>>(kt, doc_ids, row_ptr, term, val32, lens_then_ptr,
                                                                 mterm, mval);
    IVF_LAUNCH_CHECK();
  }
  return cudaSuccess;
}

cudaError_t launch_prepare_objects(int64_t n_docs, int64_t nnz, int64_t dt_local_max, const int64_t* row_ptr,
                                   const int32_t* term, int32_t* term_rebase, const float* val32, void* val_store, int storage, float* nx,
                                   int32_t n_inst, const int64_t* inst_docs, const int64_t* inst_toff,
                                   const int32_t* inst_terms, int validate, unsigned* status, unsigned* negative,
                                   cudaStream_t s) {
  (void)nnz;
  (void)dt_local_max;
  const unsigned g = grid_for(n_docs * 32, T256, 16384);
  switch (storage) {
    case ST_F16:
      k_prepare_objects<__half><<<g, T256, 0, s>>>(n_docs, row_ptr, term, term_rebase, val32, static_cast<__half*>(val_store), nx,
                                                   n_inst, inst_docs, inst_toff, inst_terms, validate, status,
                                                   negative);
      break;
    case ST_BF16:
      k_prepare_objects<__nv_bfloat16><<<g, T256, 0, s>>>(n_docs, row_ptr, term, term_rebase, val32,
                                                          static_cast<__nv_bfloat16*>(val_store), nx, n_inst,
                                                          inst_docs, inst_toff, inst_terms, validate, status,
                                                          negative);
      break;
    default:
      k_prepare_objects<float><<<g, T256, 0, s>>>(n_docs, row_ptr, term, term_rebase, val32, nullptr, nx, n_inst, inst_docs,
                                                  inst_toff, inst_terms, validate, status, negative);
      break;
  }
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_check_row_ptr(const int64_t* rp, int64_t n, int64_t nnz, unsigned* status, cudaStream_t s) {
  k_check_row_ptr<<<grid_for(n, T256, 4096), T256, 0, s>>>(rp, n, nnz, status);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

// Warp per object: scatter its head-term values into its dense row, and
// flag the (128-object block, 64-slot chunk) pairs that hold a value (every
// writer stores the same 1).
__global__ void k_build_xhead(int64_t i0, int64_t nb, const int64_t* row_ptr, const int32_t* term,
                              const uint16_t* val16, const int32_t* head_slot, uint16_t* x, int64_t ldx,
                              uint8_t* chunk_nz) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nchunks = ldx / 64;
  for (int64_t o = gw; o < nb; o += nw) {
    const int64_t i = i0 + o;
    for (int64_t h = row_ptr[i] + lane; h < row_ptr[i + 1]; h += 32) {
      const int32_t s = head_slot[term[h]];
      if (s >= 0) {
        x[o * ldx + s] = val16[h];
        if (chunk_nz != nullptr) chunk_nz[(o >> 7) * nchunks + (s >> 6)] = 1;
      }
    }
  }
}

cudaError_t launch_build_xhead(int64_t i0, int64_t nb, const int64_t* row_ptr, const int32_t* term,
                               const void* val16, const int32_t* head_slot, void* x, int64_t ldx,
                               uint8_t* chunk_nz, cudaStream_t s) {
  IVF_CU(cudaMemsetAsync(x, 0, sizeof(uint16_t) * nb * ldx, s));
  if (chunk_nz != nullptr) IVF_CU(cudaMemsetAsync(chunk_nz, 0, (size_t)((nb + 127) / 128) * (ldx / 64), s));
  k_build_xhead<<<grid_for(nb * 32, T256, 16384), T256, 0, s>>>(i0, nb, row_ptr, term,
                                                                 static_cast<const uint16_t*>(val16), head_slot,
                                                                 static_cast<uint16_t*>(x), ldx, chunk_nz);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

// 32 x 32 tiles through shared memory: wdT[c][r] = wd[r][c].
__global__ void k_transpose16(const uint16_t* __restrict__ wd, int64_t rows, int64_t kpad, uint16_t* __restrict__ wdT,
                              int64_t ldt) {
  __shared__ uint16_t tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (r < rows && c < kpad) ? wd[r * kpad + c] : (uint16_t)0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (c < kpad && r < ldt) wdT[c * ldt + r] = tile[threadIdx.x][y];
  }
}

cudaError_t launch_transpose16(const void* wd, int64_t rows, int64_t kpad, void* wdT, int64_t ldt, cudaStream_t s) {
  const dim3 grid((unsigned)((kpad + 31) / 32), (unsigned)((ldt + 31) / 32));
  k_transpose16<<<grid, dim3(32, 8), 0, s>>>(static_cast<const uint16_t*>(wd), rows, kpad,
                                             static_cast<uint16_t*>(wdT), ldt);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

}  // namespace ivfk
