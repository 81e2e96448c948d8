// Device-wide exclusive scan and stable LSD radix sort for the update step.
#include "common.cuh"
#include "radix.cuh"

namespace ivfk {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_sum(T v) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(IVF_FULL_MASK, v, o);
  if (lane == 0) warp_tot[warp] = v;
  __syncthreads();
  T t = 0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(IVF_FULL_MASK, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// Inclusive block scan; returns the inclusive prefix of v, *total = block sum.
template <typename T>
__device__ T block_inclusive(T v, T* total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(IVF_FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(IVF_FULL_MASK, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_tot[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  T add = warp > 0 ? warp_tot[warp - 1] : T(0);
  *total = warp_tot[nw - 1];
  __syncthreads();
  return x + add;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const T* in, int64_t n, T* part) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  T s = 0;
  for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_THREADS) {
    int64_t idx = base + i;
    if (idx < n) s += in[idx];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_partials(T* part, int64_t nb) {
  T carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t idx = base + threadIdx.x;
    T v = idx < nb ? part[idx] : T(0);
    T tot;
    T incl = block_inclusive(v, &tot);
    if (idx < nb) part[idx] = carry + incl - v;
    carry += tot;
  }
  if (threadIdx.x == 0) part[nb] = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const T* in, T* out, int64_t n, const T* part) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T tsum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : T(0);
    tsum += v[i];
  }
  T tot;
  T incl = block_inclusive(tsum, &tot);
  T run = part[blockIdx.x] + incl - tsum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

// The exclusive scan of 0/1 run-head flags, turned at once into the run
// starts: the r-th set flag's position goes to starts[r] (so the scanned
// flags are never written), starts[U] = n and *d_u = U, the number of runs.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_heads(const uint32_t* in, int64_t n, const uint32_t* part,
                                                             uint32_t* starts, int64_t* d_u) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t tsum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0u;
    tsum += v[i];
  }
  uint32_t tot;
  const uint32_t incl = block_inclusive(tsum, &tot);
  uint32_t run = part[blockIdx.x] + incl - tsum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (v[i] != 0u) starts[run] = (uint32_t)(base + i);
    run += v[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const uint32_t u = part[gridDim.x];
    starts[u] = (uint32_t)n;
    *d_u = (int64_t)u;
  }
}

template <typename T>
cudaError_t scan_impl(const T* in, T* out, int64_t n, void* temp, cudaStream_t s) {
  int64_t nb = ceil_div(n, SCAN_CHUNK);
  if (nb < 1) nb = 1;
  T* part = static_cast<T*>(temp);
  k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, part);
  IVF_LAUNCH_CHECK();
  k_scan_partials<T><<<1, 1024, 0, s>>>(part, nb);
  IVF_LAUNCH_CHECK();
  k_scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, part);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

// ------------------------------------------------------------ radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
// 8 keys per thread and at most 64 registers (4 blocks of 8 warps per SM):
// measured faster than 16 keys at 2 blocks per SM (more warps in flight to
// cover the load latency, a bigger but still small histogram scan)
constexpr int RS_ROUNDS = 8;
constexpr int RS_SCATTER_MIN_BLOCKS = 4;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // elements per block
constexpr int RS_BINS = 256;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const K* keys, const int64_t* d_n, int shift,
                                                           uint32_t* hist, int64_t nb) {
  __shared__ uint32_t h[RS_WARPS][RS_BINS];
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = *d_n;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const int warp = threadIdx.x >> 5;
  if (base < n) {
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
      int64_t idx = base + (int64_t)r * RS_THREADS + threadIdx.x;
      if (idx < n) atomicAdd(&h[warp][(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) c += h[w][d];
    hist[(int64_t)d * nb + blockIdx.x] = c;
  }
}

// Stable scatter of one 8-bit digit.  Each warp ranks its 8 x 32 keys with
// match_any (in input order), the block turns the per-warp counts into
// block-local positions, stages keys and values in shared memory in digit
// order, and then writes each digit's run with consecutive threads on
// consecutive addresses (coalesced), at the run's global offset.
template <typename K, typename V>
__global__ void __launch_bounds__(RS_THREADS, RS_SCATTER_MIN_BLOCKS) k_radix_scatter(const K* __restrict__ kin,
                                                              const V* __restrict__ vin,
                                                              K* __restrict__ kout, V* __restrict__ vout,
                                                              const int64_t* d_n, int shift,
                                                              const uint32_t* __restrict__ offs, int64_t nb) {
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t dbase[RS_BINS];   // global start of the block's run of digit d
  __shared__ uint32_t lbase[RS_BINS];   // block-local start of digit d
  extern __shared__ __align__(16) unsigned char rs_stage[];
  V* sv = reinterpret_cast<V*>(rs_stage);  // the wider type first: both stay aligned
  K* sk = reinterpret_cast<K*>(rs_stage + sizeof(V) * RS_TILE);
  const int64_t n = *d_n;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  if (base >= n) return;  // uniform over the block
  const int cnt = (int)(n - base < RS_TILE ? n - base : RS_TILE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  K k[RS_ROUNDS];
  V v[RS_ROUNDS];
  uint32_t rk[RS_ROUNDS];
  const int64_t wbase = base + (int64_t)warp * (RS_ROUNDS * 32);
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    const bool valid = idx < n;
    k[r] = valid ? kin[idx] : K(0);
    v[r] = valid ? vin[idx] : V(0);
    const uint32_t d = valid ? ((uint32_t)(k[r] >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(IVF_FULL_MASK, d);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (valid) before = wcnt[warp][d];
    rk[r] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && lane == leader) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: warp offsets inside the digit, and the digit's block total
  uint32_t tot = 0;
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t c = wcnt[w][d];
      wcnt[w][d] = acc;
      acc += c;
    }
    tot = acc;
    dbase[d] = offs[(int64_t)d * nb + blockIdx.x];
  }
  // block-local digit starts: exclusive scan of the totals (RS_BINS == RS_THREADS)
  {
    static_assert(RS_BINS == RS_THREADS, "one digit per thread");
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(IVF_FULL_MASK, x, o);
      if (lane >= o) x += y;
    }
    __shared__ uint32_t wsum[RS_WARPS];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += wsum[w];
    lbase[threadIdx.x] = add + x - tot;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    if (idx < n) {
      const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
      const uint32_t lp = lbase[d] + wcnt[warp][d] + rk[r];
      sk[lp] = k[r];
      sv[lp] = v[r];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
    const K key = sk[i];
    const uint32_t d = (uint32_t)(key >> shift) & 255u;
    const uint32_t pos = dbase[d] + ((uint32_t)i - lbase[d]);
    kout[pos] = key;
    vout[pos] = sv[i];
  }
}

template <typename K, typename V>
constexpr size_t scatter_smem_bytes() {
  return (sizeof(K) + sizeof(V)) * RS_TILE;
}

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

template <typename K, typename V>
cudaError_t radix_impl(K* keys, K* keys_alt, V* vals, V* vals_alt, const int64_t* d_n,
                       int64_t n_max, int bits, void* temp, cudaStream_t s, bool* in_alt) {
  int64_t nb = ceil_div(n_max, RS_TILE);
  if (nb < 1) nb = 1;
  uint32_t* hist = static_cast<uint32_t*>(temp);
  void* scan_tmp = static_cast<char*>(temp) + align_up(((size_t)RS_BINS * nb + 1) * sizeof(uint32_t));
  const int passes = (bits + 7) / 8;
  K* ki = keys;
  K* ko = keys_alt;
  V* vi = vals;
  V* vo = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_radix_hist<K><<<(unsigned)nb, RS_THREADS, 0, s>>>(ki, d_n, shift, hist, nb);
    IVF_LAUNCH_CHECK();
    IVF_CU(exclusive_scan_u32(hist, hist, (int64_t)RS_BINS * nb, scan_tmp, s));
    k_radix_scatter<K, V><<<(unsigned)nb, RS_THREADS, scatter_smem_bytes<K, V>(), s>>>(ki, vi, ko, vo, d_n,
                                                                                       shift, hist, nb);
    IVF_LAUNCH_CHECK();
    K* tk = ki;
    ki = ko;
    ko = tk;
    V* tv = vi;
    vi = vo;
    vo = tv;
  }
  *in_alt = (passes & 1) != 0;
  return cudaSuccess;
}

}  // namespace

cudaError_t radix_prepare() {
  IVF_CU(cudaFuncSetAttribute(k_radix_scatter<uint32_t, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)scatter_smem_bytes<uint32_t, uint32_t>()));
  IVF_CU(cudaFuncSetAttribute(k_radix_scatter<uint32_t, uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)scatter_smem_bytes<uint32_t, uint64_t>()));
  return cudaSuccess;
}

size_t scan_temp_bytes(int64_t n) { return ((size_t)ceil_div(n < 1 ? 1 : n, SCAN_CHUNK) + 2) * sizeof(int64_t); }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t s) {
  return scan_impl<uint32_t>(in, out, n, temp, s);
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, temp, s);
}

cudaError_t heads_to_starts(const uint32_t* flags, int64_t n, uint32_t* starts, int64_t* d_u, void* temp,
                            cudaStream_t s) {
  int64_t nb = ceil_div(n, SCAN_CHUNK);
  if (nb < 1) nb = 1;
  uint32_t* part = static_cast<uint32_t*>(temp);
  k_scan_reduce<uint32_t><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(flags, n, part);
  IVF_LAUNCH_CHECK();
  k_scan_partials<uint32_t><<<1, 1024, 0, s>>>(part, nb);
  IVF_LAUNCH_CHECK();
  k_scan_heads<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(flags, n, part, starts, d_u);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

size_t radix_temp_bytes(int64_t n_max) {
  int64_t nb = ceil_div(n_max < 1 ? 1 : n_max, RS_TILE);
  return align_up(((size_t)RS_BINS * nb + 1) * sizeof(uint32_t)) + scan_temp_bytes((int64_t)RS_BINS * nb);
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                           const int64_t* d_n, int64_t n_max, int bits, void* temp, cudaStream_t s,
                           bool* in_alt) {
  return radix_impl<uint32_t, uint32_t>(keys, keys_alt, vals, vals_alt, d_n, n_max, bits, temp, s, in_alt);
}

cudaError_t radix_sort_u32_wide(uint32_t* keys, uint32_t* keys_alt, uint64_t* vals, uint64_t* vals_alt,
                                const int64_t* d_n, int64_t n_max, int bits, void* temp, cudaStream_t s,
                                bool* in_alt) {
  return radix_impl<uint32_t, uint64_t>(keys, keys_alt, vals, vals_alt, d_n, n_max, bits, temp, s, in_alt);
}

}  // namespace ivfk
