// Assignment step of Algorithm 3 (IVF) on sm_103a, the FP64 re-score of
// near-ties, and the per-iteration reductions.
//
// Kernel design (GB300-first, not the paper's CPU loop nest):
//   * persistent grid, one warp per object, objects handed out by an atomic
//     counter (object cost sum_h (nc)_{t_(i,h)} is heavy tailed);
//   * each warp owns a private FP32 accumulator rho over a tile of the
//     cluster range in shared memory (Algorithm 3's rho in R^k, tiled when k
//     is large: per-(term, tile) offsets give each posting list's slice);
//   * the object's terms are taken one at a time and the 32 lanes stride over
//     that term's posting list xi_s: cluster ids are unique inside a list, so
//     rho_c += v * u needs no atomics, and every rho_c is summed in ascending
//     term order -- bit-reproducible from run to run and across tile shapes;
//   * argmax by a per-lane scan plus a warp butterfly on (value desc, id asc),
//     which also yields the runner-up for the top-2 gap;
//   * objects whose gap lies within the computed FP32 / FP16 / BF16 error
//     bound are queued with their candidate clusters for an FP64 re-score
//     against the FP64 master means, so the returned assignment is the FP64
//     argmax.
#include <float.h>

#include <map>
#include <mutex>

#include "assign_common.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace ivfk {

namespace {

// Drop candidates below thr (warp-cooperative, ncand uniform across lanes).
// Compaction only moves entries to lower positions, chunk by chunk.
__device__ __forceinline__ void prune_candidates(int* cand_id, float* cand_val, int& ncand, float thr, int lane) {
  int out = 0;
  for (int base = 0; base < ncand; base += 32) {
    const int q = base + lane;
    int idv = 0;
    float vv = -INFINITY;
    bool keep = false;
    if (q < ncand) {
      idv = cand_id[q];
      vv = cand_val[q];
      keep = vv >= thr;
    }
    const unsigned km = __ballot_sync(IVF_FULL_MASK, keep);
    __syncwarp();
    if (keep) {
      const int pos = out + __popc(km & ((1u << lane) - 1u));
      cand_id[pos] = idv;
      cand_val[pos] = vv;
    }
    out += __popc(km);
    __syncwarp();
  }
  ncand = out;
}

// 16 bytes of a dense head row -> floats.
template <typename WT>
__device__ __forceinline__ void unpack16(uint4 raw, float* e);
template <>
__device__ __forceinline__ void unpack16<float>(uint4 raw, float* e) {
  e[0] = __uint_as_float(raw.x);
  e[1] = __uint_as_float(raw.y);
  e[2] = __uint_as_float(raw.z);
  e[3] = __uint_as_float(raw.w);
}
template <>
__device__ __forceinline__ void unpack16<__half>(uint4 raw, float* e) {
  const uint32_t u[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __half2_raw hr;
    hr.x = (unsigned short)(u[q] & 0xFFFFu);
    hr.y = (unsigned short)(u[q] >> 16);
    const float2 f = __half22float2(__half2(hr));
    e[2 * q] = f.x;
    e[2 * q + 1] = f.y;
  }
}
template <>
__device__ __forceinline__ void unpack16<__nv_bfloat16>(uint4 raw, float* e) {
  const uint32_t u[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // a bf16 is the top half of an FP32
    e[2 * q] = __uint_as_float(u[q] << 16);
    e[2 * q + 1] = __uint_as_float(u[q] & 0xFFFF0000u);
  }
}

// R > 0: hybrid kernel.  Posting lists stored as dense head rows are
// accumulated in registers -- with VEC values per 16-byte load, lane l owns
// clusters VEC*(32g + l) + k of the tile (g < R/VEC, k < VEC; tile = 32R
// clusters) -- so they need neither cluster ids nor shared-memory
// read-modify-writes; the remaining (sparse) lists scatter into the
// shared-memory tile as in the R = 0 kernel.  Per cluster the head and the
// tail contributions are each summed in ascending term order, then added.
// SPLIT (R > 0 only): the shared-memory tile spans a.head_sub head sub-tiles;
// the sparse lists are scattered once per tile, then each sub-tile walks the
// dense rows.  Without SPLIT one pass per tile does both (head_sub == 1).
//
// Register budgets: 64 for the shared-memory kernel (1,024-thread blocks);
// the dense-head kernels hold 32R-cluster accumulators and two rows in
// flight -- 96 for FP32 rows, 128 for 16-bit rows of the 1,024-cluster tile
// (no spills; 96 would spill there).
// TC: the head part comes from the tensor-core GEMM (a.rho_head), so no dense
// rows are walked and the row registers are not needed (80 registers).
template <typename WT, int R, bool TC>
constexpr int assign_max_regs() {
  return R == 0 ? 64 : (TC ? 80 : (sizeof(WT) == 4 ? (R >= 32 ? 96 : 72) : (R >= 32 ? 128 : 96)));
}
template <typename WT, typename IdT, int R, bool SPLIT = false, bool TC = false>
__global__ void __maxnreg__((assign_max_regs<WT, R, TC>())) k_assign(const AssignArgs a) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* rho = smem + (size_t)warp * (a.tile_cap + 2 * CAND_MAX);
  int* cand_id = reinterpret_cast<int*>(rho + a.tile_cap);
  float* cand_val = rho + a.tile_cap + CAND_MAX;
  const WT* __restrict__ val = static_cast<const WT*>(a.val);
  const WT* __restrict__ w = static_cast<const WT*>(a.w);
  const IdT* __restrict__ cid = static_cast<const IdT*>(a.cid);
  const WT* __restrict__ wd = static_cast<const WT*>(a.wd);
  const int32_t* __restrict__ head_slot = a.head_slot;
  // (tensor-core head parts exist for 16-bit storage only)
  const __half* __restrict__ rho_tc = (R > 0 && TC) ? static_cast<const __half*>(a.rho_head) : nullptr;
  constexpr int RR = R > 0 ? R : 1;
  constexpr int VEC = 16 / (int)sizeof(WT);      // values per 16-byte load of a dense head row
  constexpr int NG = RR >= VEC ? RR / VEC : 1;  // 16-byte groups per lane: clusters VEC*(32g + lane) + k
  float acc[RR];
  const int cmask = a.tiled ? (a.k_tile - 1) : 0xFFFF;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long my_entries = 0, my_zero = 0;
  const bool nonneg = a.nonneg != 0 && (a.negative == nullptr || *a.negative == 0u) &&
                      (a.means_negative == nullptr || *a.means_negative == 0u);

  for (;;) {
    unsigned long long o = 0;
    if (lane == 0) o = atomicAdd(a.work, 1ull);
    o = __shfl_sync(IVF_FULL_MASK, o, 0);
    if (o >= (unsigned long long)(a.obj_list_n != nullptr ? (int64_t)*a.obj_list_n : a.n_docs)) break;
    const int64_t oi = (int64_t)o * a.obj_stride;
    int64_t i;
    int b;
    if (a.obj_list != nullptr) {
      i = a.obj_list[oi];
      b = a.n_inst > 1 ? find_instance(a.inst_docs, a.n_inst, i) : 0;
    } else if (a.obj_inst != nullptr) {
      const int q = find_instance(a.obj_prefix, a.n_obj_inst, oi);
      b = a.obj_inst[q];
      i = a.inst_docs[b] + (oi - a.obj_prefix[q]);
    } else {
      i = a.obj_base + oi;
      b = a.n_inst > 1 ? find_instance(a.inst_docs, a.n_inst, i) : 0;
    }
    const int K = a.inst_clu[b + 1] - a.inst_clu[b];
    const int64_t r0 = a.row_ptr[i], r1 = a.row_ptr[i + 1];
    const int m = (int)(r1 - r0);
    const ErrBound bound = err_bound(m, a.nx[i], a.storage, nonneg, a.rho_head != nullptr);
    const int tile = a.tiled ? a.k_tile : K;
    const int n_tiles = a.tiled ? (K + a.k_tile - 1) / a.k_tile : 1;
    if (a.tile_lo >= n_tiles) continue;  // tile-major: this object's tiles are all done
    const int tile_end = min(n_tiles, a.tile_hi);
    const bool finish = tile_end == n_tiles;
    float best = -INFINITY, second = -INFINITY;
    int bid = 0x7fffffff;
    if (a.tile_lo > 0) {  // carry of the previous tile-major launch
      best = a.best[i];
      bid = a.assign[i];
      second = a.gap[i];
    }
    int ncand = 0;
    bool overflow = false;
    const bool carry_cand = a.rescore && a.tcand != nullptr;
    if (carry_cand && a.tile_lo > 0) {  // candidates of the earlier tiles
      const int n0 = a.tcand_n[i];
      if (n0 < 0) {
        overflow = true;
      } else {
        for (int q = lane; q < n0; q += 32) {
          cand_id[q] = a.tcand[(int64_t)i * a.tcand_cap + q];
          cand_val[q] = a.tcandv[(int64_t)i * a.tcand_cap + q];
        }
        ncand = n0;
      }
      __syncwarp();
    }
    const unsigned long long entries_before = my_entries;

    // One object term per lane: its value, dense-row slot (or -1), and the
    // slice of its sparse list inside tile tt (count_head: the length of a
    // dense row's list, counted once per object for Eq. 15).
    struct TermInfo {
      float v;
      int slot;
      int64_t beg;
      int len;
    };
    auto load_term = [&](int64_t h, int tt, bool count_head) -> TermInfo {
      float v = 0.f;
      int slot = -1;
      int64_t beg = 0;
      int len = 0;
      if (h < r1) {
        const int t = __ldg(a.term + h);
        v = to_f32(val[h]);
        if (R > 0 && head_slot != nullptr) slot = __ldg(head_slot + t);
        const int64_t tb0 = __ldg(a.term_ptr + t);
        if (slot >= 0) {
          if (count_head) len = (int)(__ldg(a.term_ptr + t + 1) - tb0);
        } else if (a.tiled) {
          const int32_t* to = a.toff + (int64_t)t * (a.n_tiles_max + 1) + tt;
          const int o0 = __ldg(to), o1 = __ldg(to + 1);
          beg = tb0 + o0;
          len = o1 - o0;
        } else {
          beg = tb0;
          len = (int)(__ldg(a.term_ptr + t + 1) - tb0);
        }
      }
      return TermInfo{v, slot, beg, len};
    };
    // The sparse lists of one chunk, one at a time: rho_c += v * u.
    auto tail_scatter = [&](unsigned tm, int64_t beg, int len, float v) {
      while (tm) {
        const int j = __ffs(tm) - 1;
        tm &= tm - 1;
        const int64_t bj = __shfl_sync(IVF_FULL_MASK, beg, j);
        const int lj = __shfl_sync(IVF_FULL_MASK, len, j);
        const float vj = __shfl_sync(IVF_FULL_MASK, v, j);
        const IdT* __restrict__ cp = cid + bj;
        const WT* __restrict__ wp = w + bj;
        int q = lane;
        for (; q + 96 < lj; q += 128) {
          const int c0 = __ldg(cp + q) & cmask;
          const int c1 = __ldg(cp + q + 32) & cmask;
          const int c2 = __ldg(cp + q + 64) & cmask;
          const int c3 = __ldg(cp + q + 96) & cmask;
          const float u0 = to_f32(wp[q]);
          const float u1 = to_f32(wp[q + 32]);
          const float u2 = to_f32(wp[q + 64]);
          const float u3 = to_f32(wp[q + 96]);
          rho[c0] = fmaf(vj, u0, rho[c0]);
          rho[c1] = fmaf(vj, u1, rho[c1]);
          rho[c2] = fmaf(vj, u2, rho[c2]);
          rho[c3] = fmaf(vj, u3, rho[c3]);
        }
        for (; q < lj; q += 32) {
          const int c = __ldg(cp + q) & cmask;
          rho[c] = fmaf(vj, to_f32(wp[q]), rho[c]);
        }
        __syncwarp();
      }
    };
    // The dense head rows of one chunk, two at a time (ascending term order
    // per cluster): acc[g*VEC+k] += v * w[slo + VEC*(32g + lane) + k].
    // NR rows per round (two FP32 rows, or four 16-bit rows: the same bytes
    // in flight per lane, twice the work per round for 16-bit storage).
    constexpr int NR = sizeof(WT) == 4 ? 2 : 4;
    auto head_rows = [&](unsigned hm, int slot, float v, int slo, int ng_live) {
      if constexpr (R > 0 && NR == 2) {
        while (hm) {
          const int j0 = __ffs(hm) - 1;
          hm &= hm - 1;
          const bool two = hm != 0;
          const int j1 = two ? __ffs(hm) - 1 : j0;
          if (two) hm &= hm - 1;
          const int s0 = __shfl_sync(IVF_FULL_MASK, slot, j0);
          const int s1 = __shfl_sync(IVF_FULL_MASK, slot, j1);
          const float v0 = __shfl_sync(IVF_FULL_MASK, v, j0);
          const float v1 = two ? __shfl_sync(IVF_FULL_MASK, v, j1) : 0.f;  // fma(0, w, acc) == acc
          const uint4* __restrict__ row0 = reinterpret_cast<const uint4*>(wd + (int64_t)s0 * a.kpad + slo) + lane;
          const uint4* __restrict__ row1 = reinterpret_cast<const uint4*>(wd + (int64_t)s1 * a.kpad + slo) + lane;
          // groups that lie wholly past the sub-tile's last cluster are not
          // summed (warp-uniform); their loads stay unconditional, which keeps
          // the register count at the budget (re-pointing them at group 0 cost
          // spills and 10 % of the FP32 assignment)
          uint4 w0[NG], w1[NG];
#pragma unroll
          for (int g = 0; g < NG; ++g) w0[g] = __ldg(row0 + 32 * g);
#pragma unroll
          for (int g = 0; g < NG; ++g) w1[g] = __ldg(row1 + 32 * g);
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            if (g < ng_live) {
              float e[VEC];
              unpack16<WT>(w0[g], e);
#pragma unroll
              for (int k = 0; k < VEC; ++k) acc[g * VEC + k] = fmaf(v0, e[k], acc[g * VEC + k]);
            }
          }
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            if (g < ng_live) {
              float e[VEC];
              unpack16<WT>(w1[g], e);
#pragma unroll
              for (int k = 0; k < VEC; ++k) acc[g * VEC + k] = fmaf(v1, e[k], acc[g * VEC + k]);
            }
          }
        }
      } else if constexpr (R > 0) {
        while (hm) {
          // the next NR dense rows of the chunk, in ascending term order; a
          // missing row repeats the first with v = 0 (fma(0, w, acc) == acc)
          int sr[NR];
          float vr[NR];
          const int j0 = __ffs(hm) - 1;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const bool have = hm != 0;
            const int j = have ? __ffs(hm) - 1 : j0;
            if (have) hm &= hm - 1;
            sr[r] = __shfl_sync(IVF_FULL_MASK, slot, j);
            const float vv = __shfl_sync(IVF_FULL_MASK, v, j);
            vr[r] = have ? vv : 0.f;
          }
          // groups past the sub-tile's last cluster: not summed, loads re-read group 0
          uint4 wr[NR][NG];
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const uint4* __restrict__ row = reinterpret_cast<const uint4*>(wd + (int64_t)sr[r] * a.kpad + slo) + lane;
#pragma unroll
            for (int g = 0; g < NG; ++g) wr[r][g] = __ldg(row + 32 * (g < ng_live ? g : 0));
          }
#pragma unroll
          for (int r = 0; r < NR; ++r) {
#pragma unroll
            for (int g = 0; g < NG; ++g) {
              if (g < ng_live) {
                float e[VEC];
                unpack16<WT>(wr[r][g], e);
#pragma unroll
                for (int k = 0; k < VEC; ++k) acc[g * VEC + k] = fmaf(vr[r], e[k], acc[g * VEC + k]);
              }
            }
          }
        }
      }
    };

    // R > 0: the shared-memory tile holds head_sub head sub-tiles of 32R
    // clusters.  With one sub-tile the chunk loop does both kinds of list in
    // one pass; with several (SPLIT), the sparse lists are scattered once per
    // tile and each sub-tile then walks the object's dense rows into registers.
    constexpr bool split = R > 0 && SPLIT;
    for (int tt = a.tile_lo; tt < tile_end; ++tt) {
      const int lo = tt * tile;
      const int cnt = min(tile, K - lo);
      // rho <- 0 over the tile
      float4* r4 = reinterpret_cast<float4*>(rho);
      for (int q = lane; q < ((cnt + 3) >> 2); q += 32) r4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      __syncwarp();
      // for s in S_i (32 at a time): for (c, u) in xi_s: rho_c += v * u
      if constexpr (R == 0 || split) {
        for (int64_t h0 = r0; h0 < r1; h0 += 32) {
          const TermInfo ti0 = load_term(h0 + lane, tt, tt == 0);
          my_entries += (unsigned long long)ti0.len;
          tail_scatter(__ballot_sync(IVF_FULL_MASK, h0 + lane < r1 && ti0.slot < 0), ti0.beg, ti0.len, ti0.v);
        }
      }
      // argmax over the tile: lowest id among the maxima, plus the runner-up
      float tb = -INFINITY, ts = -INFINITY;
      int ti = 0x7fffffff;
      if constexpr (R > 0) {  // rho_c = head part (registers) + tail part (shared memory)
        constexpr int SUB = 32 * RR;
        const int nsub = split ? (cnt + SUB - 1) / SUB : 1;
        for (int sb = 0; sb < nsub; ++sb) {
          const int sbase = sb * SUB;
          const int scnt = min(SUB, cnt - sbase);
          const int ng_live = (scnt + VEC * 32 - 1) / (VEC * 32);  // 16-byte groups holding a cluster < scnt
#pragma unroll
          for (int r = 0; r < RR; ++r) acc[r] = 0.f;
          if (!split || rho_tc == nullptr) {
            for (int64_t h0 = r0; h0 < r1; h0 += 32) {
              const TermInfo ti0 = load_term(h0 + lane, tt, !split && tt == 0);
              if (!split) my_entries += (unsigned long long)ti0.len;
              if constexpr (!TC)
                head_rows(__ballot_sync(IVF_FULL_MASK, ti0.slot >= 0), ti0.slot, ti0.v, lo + sbase, ng_live);
              if (!split)
                tail_scatter(__ballot_sync(IVF_FULL_MASK, h0 + lane < r1 && ti0.slot < 0), ti0.beg, ti0.len,
                             ti0.v);
            }
          }
          if (rho_tc != nullptr) {
            // the head part from the tensor-core GEMM: same lane-to-cluster map
            const __half* __restrict__ rr = rho_tc + (i - a.obj_base) * a.rho_ld + lo + sbase;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
              if (g < ng_live) {
                float e[VEC];
                unpack16<__half>(__ldg(reinterpret_cast<const uint4*>(rr + VEC * (32 * g + lane))), e);
#pragma unroll
                for (int k = 0; k < VEC; ++k) acc[g * VEC + k] = e[k];
              }
            }
          }
          __syncwarp();
          float* rs = rho + sbase;
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            if (g >= ng_live) continue;
#pragma unroll
            for (int k4 = 0; k4 < VEC; k4 += 4) {
              const int q0 = VEC * 32 * g + VEC * lane + k4;  // 16-byte aligned, < SUB
              float4 t4 = *reinterpret_cast<const float4*>(rs + q0);
              float x[4] = {acc[g * VEC + k4] + t4.x, acc[g * VEC + k4 + 1] + t4.y, acc[g * VEC + k4 + 2] + t4.z,
                            acc[g * VEC + k4 + 3] + t4.w};
              if (q0 + 3 < scnt) {
                *reinterpret_cast<float4*>(rs + q0) = make_float4(x[0], x[1], x[2], x[3]);
#pragma unroll
                for (int k = 0; k < 4; ++k) top2_push(tb, ti, ts, x[k], lo + sbase + q0 + k);
              } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  if (q0 + k < scnt) {
                    rs[q0 + k] = x[k];
                    top2_push(tb, ti, ts, x[k], lo + sbase + q0 + k);
                  }
              }
            }
          }
          __syncwarp();
        }
      } else {
        for (int q = lane; q < cnt; q += 32) top2_push(tb, ti, ts, rho[q], lo + q);
      }
      warp_top2(tb, ti, ts);
      top2_merge(best, bid, second, tb, ti, ts);
      if (a.rescore && (a.preflag == nullptr || carry_cand)) {
        const float thr = best - bound.e2(best);
        prune_candidates(cand_id, cand_val, ncand, thr, lane);
        if (ts >= thr) {
          for (int q0 = 0; q0 < cnt; q0 += 32) {
            const int q = q0 + lane;
            const float x = q < cnt ? rho[q] : -INFINITY;
            const bool p = x >= thr;
            const unsigned pm = __ballot_sync(IVF_FULL_MASK, p);
            if (p) {
              const int pos = ncand + __popc(pm & lt);
              if (pos < CAND_MAX) {
                cand_id[pos] = lo + q;
                cand_val[pos] = x;
              }
            }
            ncand += __popc(pm);
            if (ncand > CAND_MAX) {
              overflow = true;
              ncand = CAND_MAX;
            }
          }
        } else if (tb >= thr) {
          if (ncand < CAND_MAX) {
            if (lane == 0) {
              cand_id[ncand] = ti;
              cand_val[ncand] = tb;
            }
            ++ncand;
          } else {
            overflow = true;
          }
        }
      }
      __syncwarp();
    }

    if (!finish) {  // tile-major: carry (best, id, second) and the candidates to the next launch
      if (lane == 0) {
        a.assign[i] = bid;
        a.best[i] = best;
        a.gap[i] = second;
      }
      if (carry_cand) {
        const bool over = overflow || ncand > a.tcand_cap;
        for (int q = lane; q < ncand && !over; q += 32) {
          a.tcand[(int64_t)i * a.tcand_cap + q] = cand_id[q];
          a.tcandv[(int64_t)i * a.tcand_cap + q] = cand_val[q];
        }
        if (lane == 0) a.tcand_n[i] = over ? -1 : ncand;
      }
      __syncwarp();
      continue;
    }
    const float g = best - second;
    // An object that met no posting entry has rho = 0 exactly for every
    // cluster: its lowest-id argmax is exact and needs no re-score.  A
    // tile-major launch saw only its own tiles' slices, so it asks the full
    // list lengths instead.
    bool any_entry;
    if (a.tile_lo == 0) {
      any_entry = __any_sync(IVF_FULL_MASK, my_entries != entries_before);
    } else {
      bool hit = false;
      for (int64_t h = r0 + lane; h < r1 && !hit; h += 32) {
        const int t = __ldg(a.term + h);
        hit = __ldg(a.term_ptr + t + 1) > __ldg(a.term_ptr + t);
      }
      any_entry = __any_sync(IVF_FULL_MASK, hit);
    }
    const float e2 = bound.e2(best);
    if (lane == 0) {
      a.assign[i] = bid;
      a.best[i] = best;
      a.gap[i] = g;
      if (a.err != nullptr) a.err[i] = any_entry ? 0.5f * e2 : 0.f;
      if (!any_entry) ++my_zero;
    }
    if (a.rescore && any_entry && g <= e2 && a.preflag != nullptr && (!carry_cand || overflow)) {
      // tile-major without a complete candidate list: an object-major pass
      // over these objects collects it
      if (lane == 0) a.preflag[atomicAdd(a.n_preflag, 1u)] = (int32_t)i;
    } else if (a.rescore && any_entry && g <= e2) {
      prune_candidates(cand_id, cand_val, ncand, best - e2, lane);
      unsigned slot = 0;
      if (lane == 0) slot = atomicAdd(a.n_flagged, 1u);
      slot = __shfl_sync(IVF_FULL_MASK, slot, 0);
      if ((int64_t)slot >= a.cand_slots) overflow = true;
      if (lane == 0) {
        a.flag_obj[slot] = (int32_t)i;
        a.flag_cnt[slot] = overflow ? -1 : ncand;
      }
      if (!overflow)
        for (int q = lane; q < ncand; q += 32) a.flag_cand[(int64_t)slot * CAND_MAX + q] = cand_id[q];
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_entries += __shfl_xor_sync(IVF_FULL_MASK, my_entries, o);
  if (lane == 0 && my_entries) atomicAdd(a.entries, my_entries);
  if (lane == 0 && my_zero && a.n_zero_sim != nullptr) atomicAdd(a.n_zero_sim, my_zero);
}

// ------------------------------------------------------------- re-score

__device__ __forceinline__ void top2_push_d(double& b, int& id, double& s, double x, int xid) {
  if (x > b || (x == b && xid < id)) {
    s = b;
    b = x;
    id = xid;
  } else if (x > s) {
    s = x;
  }
}

// One warp per flagged object: rho_ij in FP64 for its candidate clusters (all
// clusters on overflow) against the FP64 master means (Eq. 8): lane l sums
// the products of its terms h = l, l + 32, ... by fused multiply-add, then a
// fixed xor butterfly adds the 32 partial sums (every lane ends with the same
// bits, whatever the launch shape); then the argmax with the lowest-id tie
// rule.  A warp-serial sum in ascending h cost 32 lanes of FP64 add per
// product, and FP64 issues at a small fraction of the FP32 rate here.
__global__ void __launch_bounds__(256) k_rescore(const RescoreArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nf = (int64_t)*a.n_flagged;
  for (int64_t slot = gw; slot < nf; slot += nw) {
    const int64_t i = a.flag_obj[slot];
    const int cnt = a.flag_cnt[slot];
    const int b = a.n_inst > 1 ? find_instance(a.inst_docs, a.n_inst, i) : 0;
    const int c0 = a.inst_clu[b];
    const int K = a.inst_clu[b + 1] - c0;
    const int64_t r0 = a.row_ptr[i], r1 = a.row_ptr[i + 1];
    const int ncl = cnt < 0 ? K : cnt;
    double best = -INFINITY, second = -INFINITY;
    int bid = 0x7fffffff;
    for (int q = 0; q < ncl; ++q) {
      const int c = cnt < 0 ? q : a.flag_cand[slot * CAND_MAX + q];
      const int64_t mb = a.mptr[c0 + c], me = a.mptr[c0 + c + 1];
      double acc = 0.0;
      for (int64_t h = r0 + lane; h < r1; h += 32) {
        const int t = a.term[h];
        int64_t lo = mb, hi = me;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (a.mterm[mid] < t)
            lo = mid + 1;
          else
            hi = mid;
        }
        if (lo < me && a.mterm[lo] == t) acc = __fma_rn(f32_bits_to_f64(__float_as_uint(a.val32[h])), a.mval[lo], acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(IVF_FULL_MASK, acc, o));
      top2_push_d(best, bid, second, acc, c);
    }
    if (lane == 0) {
      const float bf = __double2float_rn(best);
      a.assign[i] = bid;
      a.best[i] = bf;
      a.gap[i] = __double2float_rn(best - second);
      // FP64 sum of at most m products in any order of additions (lane sums
      // by fused multiply-add, then the butterfly; the |v u| sum to <= ||x||):
      // (m + 1) 2^-53 ||x||, then the rounding to FP32
      if (a.err != nullptr)
        a.err[i] = fabsf(bf) * 5.9604645e-08f + (float)((double)(r1 - r0 + 1) * 1.1102230246251565e-16 *
                                                        (double)a.nx[i]) + 1e-30f;
      atomicAdd(a.n_rescored, 1ull);
    }
  }
}

// ------------------------------------------------------------ reductions

constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) k_reduce(const ReduceArgs a) {
  double obj = 0.0;
  unsigned long long ch = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_docs; i += stride) {
    const float bst = a.best[i];
    obj += (double)bst;
    const bool changed = a.prev == nullptr || a.assign[i] != a.prev[i];
    if (changed) {
      ++ch;
      if (a.n_inst > 1)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.inst_changed) + find_instance(a.inst_docs, a.n_inst, i),
                  1ull);
    }
  }
  __shared__ double so[RED_THREADS / 32];
  __shared__ unsigned long long sc[RED_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    obj += __shfl_down_sync(IVF_FULL_MASK, obj, o);
    ch += __shfl_down_sync(IVF_FULL_MASK, ch, o);
  }
  if (lane == 0) {
    so[warp] = obj;
    sc[warp] = ch;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long c = 0;
    for (int w2 = 0; w2 < RED_THREADS / 32; ++w2) {
      t += so[w2];
      c += sc[w2];
    }
    a.part_obj[blockIdx.x] = t;
    a.part_cnt[2 * blockIdx.x] = c;
  }
}

__global__ void k_reduce_final(const ReduceArgs a, int nblocks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  unsigned long long c = 0;
  for (int b = 0; b < nblocks; ++b) {
    t += a.part_obj[b];
    c += a.part_cnt[2 * b];
  }
  a.out_obj[0] = t;
  a.out_cnt[0] = c;
  a.out_cnt[1] = a.zero_sim != nullptr ? a.zero_sim[0] : 0ull;
  if (a.n_inst == 1) a.inst_changed[0] = (long long)c;
  a.acc_entries[0] += a.entries[0];
  a.acc_rescored[0] += a.n_rescored[0];
}

template <typename WT>
const void* assign_fn_r(int head_r, int head_sub, bool tc) {
  if (tc) {
    if constexpr (sizeof(WT) == 2) {
      if (head_r != HEAD_R_LARGE) return nullptr;
      return head_sub > 1 ? reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_LARGE, true, true>)
                          : reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_LARGE, false, true>);
    } else {
      return nullptr;
    }
  }
  if (head_sub > 1)
    return head_r == HEAD_R_LARGE ? reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_LARGE, true>)
           : head_r == HEAD_R_MID ? reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_MID, true>)
                                  : nullptr;
  switch (head_r) {
    case HEAD_R_SMALL:
      return reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_SMALL>);
    case HEAD_R_MID:
      return reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_MID>);
    case HEAD_R_LARGE:
      return reinterpret_cast<const void*>(&k_assign<WT, uint16_t, HEAD_R_LARGE>);
    default:
      return reinterpret_cast<const void*>(&k_assign<WT, uint16_t, 0>);
  }
}

const void* assign_fn_for(int storage, int head_r, int head_sub, bool tc) {
  switch (storage) {
    case ST_F16:
      return assign_fn_r<__half>(head_r, head_sub, tc);
    case ST_BF16:
      return assign_fn_r<__nv_bfloat16>(head_r, head_sub, tc);
    default:
      return assign_fn_r<float>(head_r, head_sub, tc);
  }
}

template <typename WT>
void launch_typed(const AssignArgs& a, int warps, int blocks, size_t smem, cudaStream_t s, int head_r) {
  if constexpr (sizeof(WT) == 2) {
    if (a.rho_head != nullptr) {  // tensor-core head (head_r == HEAD_R_LARGE, checked by the caller)
      if (a.head_sub > 1)
        k_assign<WT, uint16_t, HEAD_R_LARGE, true, true><<<blocks, warps * 32, smem, s>>>(a);
      else
        k_assign<WT, uint16_t, HEAD_R_LARGE, false, true><<<blocks, warps * 32, smem, s>>>(a);
      return;
    }
  }
  if (head_r == HEAD_R_LARGE && a.head_sub > 1) {
    k_assign<WT, uint16_t, HEAD_R_LARGE, true><<<blocks, warps * 32, smem, s>>>(a);
    return;
  }
  if (head_r == HEAD_R_MID && a.head_sub > 1) {
    k_assign<WT, uint16_t, HEAD_R_MID, true><<<blocks, warps * 32, smem, s>>>(a);
    return;
  }
  switch (head_r) {
    case HEAD_R_SMALL:
      k_assign<WT, uint16_t, HEAD_R_SMALL><<<blocks, warps * 32, smem, s>>>(a);
      break;
    case HEAD_R_MID:
      k_assign<WT, uint16_t, HEAD_R_MID><<<blocks, warps * 32, smem, s>>>(a);
      break;
    case HEAD_R_LARGE:
      k_assign<WT, uint16_t, HEAD_R_LARGE><<<blocks, warps * 32, smem, s>>>(a);
      break;
    default:
      k_assign<WT, uint16_t, 0><<<blocks, warps * 32, smem, s>>>(a);
      break;
  }
}

}  // namespace

size_t assign_smem_bytes(int tile_cap, int warps) {
  return (size_t)warps * ((size_t)tile_cap + 2 * CAND_MAX) * sizeof(float);
}

// The shared-memory opt-in of a kernel is process-wide, so it only ever grows:
// a context with a smaller tile must not lower it under another's launches.
cudaError_t assign_prepare(int storage, int tile_cap, int warps, int head_r, int head_sub, bool tc) {
  static std::mutex mu;
  static std::map<const void*, size_t> raised;
  const size_t bytes = assign_smem_bytes(tile_cap, warps);
  const void* fn = assign_fn_for(storage, head_r, head_sub, tc);
  if (fn == nullptr) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = raised[fn];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int assign_max_blocks_per_sm(int storage, int tile_cap, int warps, int head_r, int head_sub, bool tc) {
  int nb = 0;
  if (assign_prepare(storage, tile_cap, warps, head_r, head_sub, tc) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, assign_fn_for(storage, head_r, head_sub, tc), warps * 32,
                                                    assign_smem_bytes(tile_cap, warps)) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_assign(const AssignArgs& a, int warps, int blocks, cudaStream_t s, int head_r) {
  if ((a.tiled && a.toff == nullptr) || (head_r > 0 && (a.head_slot == nullptr || a.wd == nullptr)) ||
      a.head_sub < 1 || (a.head_sub > 1 && head_r != HEAD_R_LARGE && head_r != HEAD_R_MID) ||
      (a.rho_head != nullptr && (head_r != HEAD_R_LARGE || a.storage == ST_F32)))
    return cudaErrorInvalidValue;
  const size_t smem = assign_smem_bytes(a.tile_cap, warps);
  switch (a.storage) {
    case ST_F16:
      launch_typed<__half>(a, warps, blocks, smem, s, head_r);
      break;
    case ST_BF16:
      launch_typed<__nv_bfloat16>(a, warps, blocks, smem, s, head_r);
      break;
    default:
      launch_typed<float>(a, warps, blocks, smem, s, head_r);
      break;
  }
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t assign_prepare_i32ids(int tile_cap, int warps) {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_assign<float, int32_t, 0>),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assign_smem_bytes(tile_cap, warps));
}

int assign_max_blocks_per_sm_i32ids(int tile_cap, int warps) {
  int nb = 0;  // the shared-memory limit was raised once at set-up (assign_prepare_i32ids)
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, reinterpret_cast<const void*>(&k_assign<float, int32_t, 0>),
                                                    warps * 32, assign_smem_bytes(tile_cap, warps)) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_assign_i32ids(const AssignArgs& a, int warps, int blocks, cudaStream_t s) {
  k_assign<float, int32_t, 0><<<blocks, warps * 32, assign_smem_bytes(a.tile_cap, warps), s>>>(a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_rescore(const RescoreArgs& a, int blocks, cudaStream_t s) {
  k_rescore<<<blocks, 256, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_reduce(const ReduceArgs& a, int blocks, cudaStream_t s) {
  k_reduce<<<blocks, RED_THREADS, 0, s>>>(a);
  IVF_LAUNCH_CHECK();
  k_reduce_final<<<1, 32, 0, s>>>(a, blocks);
  IVF_LAUNCH_CHECK();
  return cudaSuccess;
}

}  // namespace ivfk
