// Tensor-core head for FP16/BF16 storage, hand-written for sm_103a
// (tcgen05 MMA with TMEM accumulators, operands staged by TMA).
//
// The dense head block is the paper's full inverted file IFN (Section 4)
// restricted to the terms whose posting lists are dense: for a batch of
// objects, the head part of every similarity is
//     rho_h[i][c] = sum_s  x_h[i][s] * w_h[c][s]
// with x_h the objects' values at the head terms (slot s of term t) and w_h
// the means' values there.  That is a plain dense contraction, so it runs on
// the 5th-generation tensor cores:
//   * A = x_h (batch x T, K-major) and B = w_h (kpad x T, K-major), 16-bit,
//     staged into shared memory by TMA (cp.async.bulk.tensor, 128-byte
//     swizzle) through a 3-stage mbarrier ring of 256-object x 64-slot A
//     tiles and 256-cluster x 64-slot B tiles;
//   * one elected thread issues tcgen05.mma (M = 128 objects, N = 256
//     clusters, K = 16 per instruction) for both 128-object halves of the
//     256-object tile against the same B stage -- half the B traffic per
//     flop of a 128-object tile -- into two FP32 accumulators in TMEM (512
//     columns);
//   * eight epilogue warps read the accumulators with tcgen05.ld and store
//     them as FP16 for the assignment (which adds the sparse tail and takes
//     the argmax), or in the operands' type for ivf_head_product;
//   * a K-chunk of 64 head slots that is zero for all 256 objects of a tile
//     (flags from the kernel that builds x_h, per 128 objects) is neither
//     loaded nor multiplied;
//   * persistent grid, one CTA per SM, tiles in bands of 32 object blocks so
//     that a band's A rows and the B slices in use stay in L2.
// Every wait on an mbarrier is bounded (about two seconds of the global
// timer): on expiry the CTA raises a status bit, lets its copies and MMAs in
// flight finish, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/ivf.h"
#include "common.cuh"
#include "kernels.cuh"

namespace ivfk {

namespace {

constexpr int HM = 128;      // objects per MMA = TMEM lanes
constexpr int BM = 2 * HM;   // objects per tile: two MMA halves over one B stage
constexpr int BN = 256;      // clusters per tile = TMEM columns of one accumulator
constexpr int BK = 64;       // head slots per stage: 128 bytes of 16-bit values = one swizzle row
constexpr int STAGES = 3;
constexpr int UK = 16;       // K of one tcgen05.mma for 16-bit operands
constexpr int A_BYTES = BM * BK * 2;
constexpr int A_HALF_BYTES = HM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * BN;  // accumulator of half h at columns h * BN
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int BAND = 32;      // object blocks per band of the tile order
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

struct TcArgs {
  int64_t m;                // objects in the batch: rows of A and of D
  int32_t n;                // clusters: rows of B, columns of D (multiple of BN)
  int32_t k;                // head slots (multiple of BK)
  uint16_t* d;              // [m x ldd] in the storage type
  int64_t ldd;
  uint32_t idesc;           // instruction descriptor
  const uint8_t* chunk_nz;  // [ceil(m / HM) x k / BK] nonzero flags per 128 objects, or null (all chunks)
  unsigned* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false when the wait
// ran out of time or another role of the CTA gave up (abort flag).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  const unsigned long long t0 = now_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort) return false;
      if (now_ns() - t0 > WAIT_NS) {
        *abort = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzle layout TMA writes: rows of 128 bytes, 8-row groups 1,024 bytes
// apart (stride byte offset); the leading byte offset is unused for this
// layout; bits 46-48 hold the descriptor version 1; layout 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// Arrive on bar once every tcgen05 operation this thread issued so far is done.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tile_coords(int64_t t, int m_blocks, int n_blocks, int* mb, int* nb) {
  const int64_t per_band = (int64_t)BAND * n_blocks;
  const int64_t band = t / per_band;
  const int64_t r = t % per_band;
  const int64_t m0 = band * BAND;
  const int64_t rows = (m_blocks - m0) < BAND ? (m_blocks - m0) : BAND;  // last band may be short
  *mb = (int)(m0 + r % rows);
  *nb = (int)(r / rows);
}

// chunk kc of 256-object tile mb holds a value (either 128-object half)
__device__ __forceinline__ bool chunk_live(const TcArgs& a, int mb, int kc, int kchunks) {
  if (a.chunk_nz == nullptr) return true;
  const int64_t h0 = 2 * (int64_t)mb;
  const int64_t nh = (a.m + HM - 1) / HM;
  return a.chunk_nz[h0 * kchunks + kc] != 0 || (h0 + 1 < nh && a.chunk_nz[(h0 + 1) * kchunks + kc] != 0);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) {
  const float a = __uint_as_float(lo), b = __uint_as_float(hi);
  if constexpr (BF16) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&p);
  } else {
    const __half2 p = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&p);
  }
}

// BF16: the output type (the operand type is in the instruction descriptor
// and the tensor maps).
template <bool BF16>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_head(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sa = smem;
  uint8_t* sb = smem + STAGES * A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // full[STAGES], empty[STAGES], acc_full, acc_empty, drain
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t accf = smem_u32(bars + 2 * STAGES), acce = smem_u32(bars + 2 * STAGES + 1);
  const uint32_t drain = smem_u32(bars + 2 * STAGES + 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 3);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_blocks = (int)((a.m + BM - 1) / BM), n_blocks = a.n / BN, kchunks = a.k / BK;
  const int64_t n_tiles = (int64_t)m_blocks * n_blocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, EPI_WARPS);  // one arrival per epilogue warp
    mbar_init(drain, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      uint32_t stage = 0, phase = 0;
      uint32_t issued = 0;  // stages with a copy issued (for the drain on abort)
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        int mb, nb;
        tile_coords(t, m_blocks, n_blocks, &mb, &nb);
        for (int kc = 0; kc < kchunks; ++kc) {
          if (!chunk_live(a, mb, kc, kchunks)) continue;
          if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full0 + 8 * stage, STAGE_BYTES);
          tma_load_2d(smem_u32(sa + stage * A_BYTES), &map_a, kc * BK, mb * BM, full0 + 8 * stage);
          tma_load_2d(smem_u32(sb + stage * B_BYTES), &map_b, kc * BK, nb * BN, full0 + 8 * stage);
          issued |= 1u << stage;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // let every copy in flight land before the CTA's shared memory goes away:
        // the last copy into stage s completed the phase that precedes `phase`
        // there (or `phase ^ 1` for the stages before the current one)
        for (uint32_t s = 0; s < STAGES; ++s) {
          if (!(issued >> s & 1u)) continue;
          const uint32_t par = s < stage ? phase : (phase ^ 1u);
          const unsigned long long t0 = now_ns();
          while (!mbar_try_wait(full0 + 8 * s, par) && now_ns() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t stage = 0, phase = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        int mb, nb;
        tile_coords(t, m_blocks, n_blocks, &mb, &nb);
        if (!mbar_wait(acce, acc_phase ^ 1u, abort)) break;  // the epilogue has drained the accumulators
        fence_after_sync();
        uint32_t accumulate = 0;
        for (int kc = 0; kc < kchunks; ++kc) {
          if (!chunk_live(a, mb, kc, kchunks)) continue;
          if (!mbar_wait(full0 + 8 * stage, phase, abort)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t a0 = smem_u32(sa + stage * A_BYTES), b0 = smem_u32(sb + stage * B_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / UK; ++kk) {
            const uint64_t bd = sw128_desc(b0 + kk * UK * 2);
            umma(tmem, sw128_desc(a0 + kk * UK * 2), bd, a.idesc, accumulate);
            umma(tmem + BN, sw128_desc(a0 + A_HALF_BYTES + kk * UK * 2), bd, a.idesc, accumulate);
            accumulate = 1;
          }
          umma_commit(empty0 + 8 * stage);  // the stage is free once these MMAs have read it
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(accf);  // accumulators complete (immediately when no chunk was live)
        acc_phase ^= 1u;
      }
      // every MMA issued has finished before the TMEM is freed
      umma_commit(drain);
      const unsigned long long t0 = now_ns();
      while (!mbar_try_wait(drain, 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else {  // epilogue: warps 2-9; TMEM lane quarter warp % 4, M half (warp - 2) / 4
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = half * HM + q * 32 + lane;
    uint32_t acc_phase = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      int mb, nb;
      tile_coords(t, m_blocks, n_blocks, &mb, &nb);
      if (!mbar_wait(accf, acc_phase, abort)) break;
      fence_after_sync();
      bool live = a.chunk_nz == nullptr;
      for (int kc = 0; kc < kchunks && !live; ++kc) live = chunk_live(a, mb, kc, kchunks);
      const int64_t gm = (int64_t)mb * BM + row;
      uint16_t* drow = a.d + gm * a.ldd + (int64_t)nb * BN;
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        uint32_t v[32];
        if (live) {
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + half * BN + c, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        if (gm < a.m) {
          uint4* dst = reinterpret_cast<uint4*>(drow + c);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dst[j] = make_uint4(pack2<BF16>(v[8 * j], v[8 * j + 1]), pack2<BF16>(v[8 * j + 2], v[8 * j + 3]),
                                pack2<BF16>(v[8 * j + 4], v[8 * j + 5]), pack2<BF16>(v[8 * j + 6], v[8 * j + 7]));
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce);
      acc_phase ^= 1u;
    }
  }
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicOr(a.status, STS_TIMEOUT);
  if (warp == 1) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B type (bits 7-9, 10-12: 0 = F16, 1 = BF16), both K-major
// (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
uint32_t make_idesc(bool bf16) {
  const uint32_t ab = bf16 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(HM >> 4) << 24);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D tensor map of a row-major [rows x cols] 16-bit matrix, box [box_rows x 64].
bool encode_2d(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld_elems, int box_rows,
               bool bf16) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (fn == nullptr) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_elems * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_tc_head(const TcHeadArgs& h, cudaStream_t s) {
  if (h.m < 1 || h.n < BN || h.n % BN != 0 || h.k < BK || h.k % BK != 0 || h.lda % 8 != 0 || h.ldb % 8 != 0 ||
      h.ldd % 8 != 0 || h.lda < h.k || h.ldb < h.k || h.ldd < h.n ||
      (reinterpret_cast<uintptr_t>(h.a) & 15u) != 0 || (reinterpret_cast<uintptr_t>(h.b) & 15u) != 0 ||
      (reinterpret_cast<uintptr_t>(h.d) & 15u) != 0)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!encode_2d(&ma, h.a, h.m, h.k, h.lda, BM, h.bf16) || !encode_2d(&mb, h.b, h.n, h.k, h.ldb, BN, h.bf16))
    return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tc_head<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_tc_head<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  });
  if (attr != cudaSuccess) return attr;
  TcArgs a;
  a.m = h.m;
  a.n = h.n;
  a.k = h.k;
  a.d = static_cast<uint16_t*>(h.d);
  a.ldd = h.ldd;
  a.idesc = make_idesc(h.bf16);  // the operand type; the output type is the kernel's template argument
  a.chunk_nz = h.chunk_nz;
  a.status = h.status;
  const int64_t tiles = ((h.m + BM - 1) / BM) * (h.n / BN);
  const int grid = (int)(tiles < h.num_sms ? tiles : h.num_sms);
  if (h.out_bf16)
    k_tc_head<true><<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, a);
  else
    k_tc_head<false><<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

}  // namespace ivfk

namespace {
__device__ unsigned g_head_product_status;  // STS_TIMEOUT of the last ivf_head_product call
}  // namespace

// C ABI: the tensor-core head product on caller buffers (include/ivf.h).
extern "C" ivf_status ivf_head_product(int64_t m, int32_t n, int32_t k, const void* a, int64_t lda, const void* b,
                                       int64_t ldb, void* d, int64_t ldd, int32_t storage, void* cuda_stream) {
  if (storage != IVF_F16 && storage != IVF_BF16) return IVF_E_INVALID;
  if (!a || !b || !d) return IVF_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return IVF_E_CUDA;
  unsigned* st = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&st), g_head_product_status) != cudaSuccess) return IVF_E_CUDA;
  if (cudaMemsetAsync(st, 0, sizeof(unsigned), s) != cudaSuccess) return IVF_E_CUDA;
  ivfk::TcHeadArgs h;
  h.m = m;
  h.n = n;
  h.k = k;
  h.a = a;
  h.lda = lda;
  h.b = b;
  h.ldb = ldb;
  h.d = d;
  h.ldd = ldd;
  h.bf16 = storage == IVF_BF16;
  h.out_bf16 = h.bf16;
  h.chunk_nz = nullptr;
  h.status = st;
  h.num_sms = sms;
  const cudaError_t e = ivfk::launch_tc_head(h, s);
  if (e == cudaErrorInvalidValue) return IVF_E_INVALID;
  if (e != cudaSuccess) return IVF_E_CUDA;
  unsigned hs = 0;
  if (cudaMemcpyAsync(&hs, st, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return IVF_E_CUDA;
  return (hs & ivfk::STS_TIMEOUT) ? IVF_E_TIMEOUT : IVF_OK;
}
