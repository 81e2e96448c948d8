// Device helpers shared by the assignment kernels (assign.cu, ivfd.cu):
// the lowest-id top-2 of similarities and the error bound that decides the
// FP64 re-score of near-ties.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ivfk {

// Push similarity x of cluster xid into (best b of id, second s).  Every
// caller pushes one thread's clusters in ascending id, so a tie keeps the
// earlier, lower id and only a strictly larger x takes the best place
// (branch-free: three selects and a max).
__device__ __forceinline__ void top2_push(float& b, int& id, float& s, float x, int xid) {
  const bool gt = x > b;
  s = gt ? b : fmaxf(s, x);
  id = gt ? xid : id;
  b = gt ? x : b;
}

__device__ __forceinline__ void top2_merge(float& b, int& id, float& s, float b2, int id2, float s2) {
  if (b2 > b || (b2 == b && id2 < id)) {
    s = fmaxf(s2, b);
    b = b2;
    id = id2;
  } else {
    s = fmaxf(s, b2);
  }
}

__device__ __forceinline__ void warp_top2(float& b, int& id, float& s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float b2 = __shfl_xor_sync(IVF_FULL_MASK, b, o);
    const int id2 = __shfl_xor_sync(IVF_FULL_MASK, id, o);
    const float s2 = __shfl_xor_sync(IVF_FULL_MASK, s, o);
    top2_merge(b, id, s, b2, id2, s2);
  }
}

__device__ __forceinline__ int find_instance(const int64_t* offs, int n_inst, int64_t x) {
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

// Upper bound on |rho_hat - rho| for one object against any unit mean, where
// rho is exact with the FP64 master mean and rho_hat the FP32 accumulation of
// the stored (rounded) values.  m = number of object terms (>= number of
// products summed into any rho_c), nx >= ||x||_2.
//   FP32: mean rounding u*S plus FMA recursive summation gamma_m * S(1+u).
//   FP16/BF16: both operands rounded (u' = u16 + 2u for the FP64->FP32->16
//   double rounding), products exact in FP32, plus the FP16 subnormal floor
//   and gamma_m on the summed magnitudes.
//   With every object value and mean value >= 0 the products are all >= 0,
//   so sum_h |v u| is rho itself and the bound scales with the similarity:
//   E(rho_hat) = rel * rho_hat + abs (P = exact sum of the stored products,
//   c = per-product relative error: |rho_hat - P| <= gamma P,
//   |P - rho| <= c rho + sub, rho <= (P + sub)/(1 - c), P <= rho_hat/(1 - gamma)).
//   Otherwise E is the constant S-based bound (rel = 0).
struct ErrBound {
  float rel, abs;
  __device__ __forceinline__ float e2(float rho_hat) const { return 2.f * (rel * fmaxf(rho_hat, 0.f) + abs); }
};

__device__ __forceinline__ ErrBound err_bound(int m, float nx, int storage, bool nonneg, bool tc_head) {
  const float u32 = 5.9604645e-08f;  // 2^-24
  const float fm = (float)m;
  // m + 1 roundings at most per rho_c: up to m FMAs in the head and tail
  // chains together, plus the one addition that joins them.  A head part
  // summed by tensor cores is charged 2^-22 per addition (their FP32
  // accumulation is not specified as round-to-nearest).
  const float ua = tc_head ? 4.f * u32 : u32;
  const float g = (fm + 1.f) * ua / (1.f - (fm + 1.f) * ua);
  float c, sub;
  if (storage == ST_F32) {
    c = u32;           // the mean's rounding to FP32; object values are exact
    sub = fm * 1e-37f;  // FP32 subnormal floor (negligible)
  } else {
    const float u16 = storage == ST_F16 ? 4.8828125e-04f : 3.90625e-03f;
    const float up = u16 + 2.f * u32;
    c = 2.f * up + up * up;
    sub = storage == ST_F16 ? fm * u32 * (1.f + up) : fm * 1e-37f;
    // a tensor-core head part arrives rounded to FP16 (for either storage
    // type): one more relative 2^-11 on the head products' sum
    // (|H| <= sum of |v u| there) and half the FP16 subnormal spacing
    if (tc_head) {
      c += 4.8828125e-04f;
      sub += 2.9802322e-08f;
    }
  }
  ErrBound b;
  if (nonneg) {
    b.rel = (g + c / (1.f - c)) / (1.f - g) * 1.0001f;
    b.abs = sub / (1.f - c) * 1.0001f;
  } else {
    const float S = nx * 1.000001f;
    float e;
    if (storage == ST_F32)
      e = S * (u32 + g * (1.f + u32));
    else
      e = S * c + sub + g * (S * (1.f + c) + sub);
    b.rel = 0.f;
    b.abs = e * 1.0001f;
  }
  return b;
}

}  // namespace ivfk
