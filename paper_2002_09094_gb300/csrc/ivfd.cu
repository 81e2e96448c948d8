// IVFD (Algorithm 4, Section 7.2) on sm_103a: the assignment step with the
// inverted file on the OBJECT side, as the measured comparison with IVF.
//
// The paper's IVFD keeps the objects twice: in the standard sparse form (for
// the update step, as IVF does) and as an inverted file zeta -- for every
// term s the list of (object o, value u) in ascending o.  Its assignment
// loops over the means: for each mean mu_j and each of its terms s, every
// entry (o, u) of zeta_s adds v' * u to rho_o; after the mean, every object
// compares rho_o with its best so far.  Same multiplications as IVF (Eq. 15),
// in the transposed loop order; the paper predicts it is slower when N >> k.
//
// GPU form: the object range is cut into sub-ranges of IVFD_SUB objects and
// the means into chunks; one warp owns (sub-range, chunk) with an FP32
// accumulator per object of its sub-range in shared memory.  Per (term,
// sub-range) offsets into zeta (zoff, built once per object set) give each
// list's slice.  The mean's terms are taken 32 at a time and their non-empty
// slices scattered one after another (object ids are unique inside a list),
// so every rho_o is summed in ascending term order: the same FP32 operations
// as the sparse IVF kernel, hence the same bits.  A warp keeps the top-2 of
// its chunk per object (lowest id on ties); a merge kernel combines the
// chunks, then finishes each object as the IVF kernel does (gap, error bound,
// zero-similarity count; near-ties handed to an object-major IVF pass that
// collects their candidate clusters for the FP64 re-score).
#include "assign_common.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace ivfk {

namespace {

constexpr int T256 = 256;
constexpr int IVFD_WARPS = 4;  // 4 x 4 arrays x IVFD_SUB floats of shared memory = 32 KB

unsigned grid_of(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t g = ceil_div(n < 1 ? 1 : n, threads);
  if (g > cap) g = cap;
  return (unsigned)g;
}

// first position in a zeta list whose object is >= o
__device__ __forceinline__ int64_t lower_bound_obj(const uint64_t* a, int64_t n, int64_t o) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)(a[mid] >> 32) < o)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// zoff[s * (R + 1) + r] = offset in zeta_s of its first object >= r * SUB
__global__ void k_z_off(const IvfdArgs a) {
  const int64_t per = a.n_sub + 1;
  const int64_t total = a.dt * per;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
    const int64_t s = x / per, r = x % per;
    const int64_t b = a.zptr[s], n = a.zptr[s + 1] - b;
    const int64_t o = r * IVFD_SUB;
    a.zoff[x] = (int32_t)(o >= a.n_docs ? n : lower_bound_obj(a.zov + b, n, o));
  }
}

// One warp per (sub-range r, mean chunk c): warp index w = c * R + r, so the
// warps running together share the same means in L2.
__global__ void __launch_bounds__(IVFD_WARPS * 32) k_ivfd(const IvfdArgs a) {
  __shared__ float s_rho[IVFD_WARPS][IVFD_SUB];
  __shared__ float s_best[IVFD_WARPS][IVFD_SUB];
  __shared__ float s_second[IVFD_WARPS][IVFD_SUB];
  __shared__ int s_id[IVFD_WARPS][IVFD_SUB];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * IVFD_WARPS + wl;
  if (w >= a.n_sub * a.chunks) return;
  const int64_t r = w % a.n_sub, c = w / a.n_sub;
  const int64_t o0 = r * IVFD_SUB;
  const int ns = (int)min((int64_t)IVFD_SUB, a.n_docs - o0);
  const int j0 = (int)((int64_t)a.k * c / a.chunks), j1 = (int)((int64_t)a.k * (c + 1) / a.chunks);
  float* rho = s_rho[wl];
  float* bb = s_best[wl];
  float* ss = s_second[wl];
  int* ii = s_id[wl];
  for (int m = lane; m < IVFD_SUB; m += 32) {
    rho[m] = 0.f;
    bb[m] = -INFINITY;
    ss[m] = -INFINITY;
    ii[m] = 0x7fffffff;
  }
  __syncwarp();
  const int64_t per = a.n_sub + 1;
  unsigned long long my_entries = 0;
  for (int j = j0; j < j1; ++j) {
    const int64_t mb = a.mptr[j], me = a.mptr[j + 1];
    for (int64_t h0 = mb; h0 < me; h0 += 32) {
      const int64_t h = h0 + lane;
      float v = 0.f;
      int64_t beg = 0;
      int len = 0;
      if (h < me) {
        const int32_t s = a.mterm[h];
        v = __double2float_rn(a.mval[h]);  // the FP32 value IVF's inverted file holds
        const int32_t* zo = a.zoff + (int64_t)s * per + r;
        const int lo = __ldg(zo), hi = __ldg(zo + 1);
        beg = __ldg(a.zptr + s) + lo;
        len = hi - lo;
      }
      my_entries += (unsigned long long)len;
      unsigned tm = __ballot_sync(IVF_FULL_MASK, len > 0);
      while (tm) {
        const int q = __ffs(tm) - 1;
        tm &= tm - 1;
        const int64_t bq = __shfl_sync(IVF_FULL_MASK, beg, q);
        const int lq = __shfl_sync(IVF_FULL_MASK, len, q);
        const float vq = __shfl_sync(IVF_FULL_MASK, v, q);
        for (int e = lane; e < lq; e += 32) {
          const uint64_t ov = __ldg(a.zov + bq + e);
          const int o = (int)(ov >> 32) - (int)o0;
          rho[o] = fmaf(vq, __uint_as_float((uint32_t)ov), rho[o]);
        }
        __syncwarp();
      }
    }
    // Algorithm 4's per-mean comparison: every object of the sub-range
    for (int m = lane; m < ns; m += 32) {
      top2_push(bb[m], ii[m], ss[m], rho[m], j);
      rho[m] = 0.f;
    }
    __syncwarp();
  }
  const int64_t base = c * a.n_docs + o0;
  for (int m = lane; m < ns; m += 32) {
    a.pbest[base + m] = bb[m];
    a.psecond[base + m] = ss[m];
    a.pid[base + m] = ii[m];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_entries += __shfl_xor_sync(IVF_FULL_MASK, my_entries, o);
  if (lane == 0 && my_entries) atomicAdd(a.entries, my_entries);
}

// Warp per object: merge the chunks' top-2 in chunk order, then finish the
// object as the IVF kernel does.
__global__ void k_ivfd_finish(const IvfdArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool nonneg = a.nonneg != 0 && (a.negative == nullptr || *a.negative == 0u) &&
                      (a.means_negative == nullptr || *a.means_negative == 0u);
  unsigned long long my_zero = 0;
  for (int64_t i = gw; i < a.n_docs; i += nw) {
    float best = -INFINITY, second = -INFINITY;
    int bid = 0x7fffffff;
    for (int c = 0; c < a.chunks; ++c) {
      const int64_t x = (int64_t)c * a.n_docs + i;
      top2_merge(best, bid, second, a.pbest[x], a.pid[x], a.psecond[x]);
    }
    const int64_t r0 = a.row_ptr[i], r1 = a.row_ptr[i + 1];
    bool hit = false;
    for (int64_t h = r0 + lane; h < r1 && !hit; h += 32) {
      const int t = a.term[h];
      hit = a.term_ptr[t + 1] > a.term_ptr[t];
    }
    const bool any_entry = __any_sync(IVF_FULL_MASK, hit);
    const ErrBound bound = err_bound((int)(r1 - r0), a.nx[i], ST_F32, nonneg, false);
    const float g = best - second;
    const float e2 = bound.e2(best);
    if (lane == 0) {
      a.assign[i] = bid;
      a.best[i] = best;
      a.gap[i] = g;
      if (a.err != nullptr) a.err[i] = any_entry ? 0.5f * e2 : 0.f;
      if (!any_entry) ++my_zero;
      if (a.rescore && any_entry && g <= e2) {
        if (a.preflag != nullptr) {  // candidates collected by an IVF pass over the near-ties
          a.preflag[atomicAdd(a.n_preflag, 1u)] = (int32_t)i;
        } else {  // FP64 re-score against every cluster
          const unsigned slot = atomicAdd(a.n_flagged, 1u);
          a.flag_obj[slot] = (int32_t)i;
          a.flag_cnt[slot] = -1;
        }
      }
    }
  }
  if (lane == 0 && my_zero && a.n_zero_sim != nullptr) atomicAdd(a.n_zero_sim, my_zero);
}

}  // namespace

int64_t ivfd_sub_ranges(int64_t n_docs) { return ceil_div(n_docs, IVFD_SUB); }

cudaError_t launch_build_ivfd_offsets(const IvfdArgs& a, cudaStream_t s) {
  k_z_off<<<grid_of(a.dt * (a.n_sub + 1), T256, 65536), T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_assign_ivfd(const IvfdArgs& a, cudaStream_t s) {
  if (a.n_docs < 1 || a.chunks < 1 || a.k < 1) return cudaErrorInvalidValue;
  const int64_t warps = a.n_sub * a.chunks;
  k_ivfd<<<(unsigned)ceil_div(warps, IVFD_WARPS), IVFD_WARPS * 32, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  k_ivfd_finish<<<grid_of(a.n_docs * 32, T256, 16384), T256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

}  // namespace ivfk
