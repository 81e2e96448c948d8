// Device-wide exclusive scan and stable LSD radix sort (key, uint32 payload).
//
// These are the counting-sort and prefix-sum building blocks of the update
// step: grouping objects by cluster (the sets C_j of Algorithm 3), grouping
// the objects' term-major tuples by cluster for the member sums, the
// term-major copy of the objects itself, and the term-major rebuild of the inverted file
// (Section 3: each posting list xi_s ascends in cluster id because a stable
// sort by term keeps the cluster-major input order).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ivfk {

// Exclusive scan of n values into out[0..n]; out[n] receives the total.
// in and out may be the same array (out must hold n+1 values).
size_t scan_temp_bytes(int64_t n);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t s);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* temp, cudaStream_t s);
// n flags of 0 or 1 (run heads) -> starts[r] = position of the r-th head,
// starts[U] = n, *d_u = U (starts must hold n + 1 values).
cudaError_t heads_to_starts(const uint32_t* flags, int64_t n, uint32_t* starts, int64_t* d_u, void* temp,
                            cudaStream_t s);

// Stable LSD radix sort of d_n[0] (<= n_max) pairs, 8 bits per pass over the
// low `bits` bits of the key.  Buffers ping-pong between (keys, vals) and
// (keys_alt, vals_alt); *in_alt reports where the result ends up (a function
// of `bits` only, so it is the same at every graph replay).
// radix_prepare() opts the scatter kernels in to their shared-memory staging
// area; call it once per process (per device) before the first sort.
size_t radix_temp_bytes(int64_t n_max);
cudaError_t radix_prepare();
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                           const int64_t* d_n, int64_t n_max, int bits, void* temp, cudaStream_t s,
                           bool* in_alt);
// The same with 64-bit payloads (carried through every pass).
cudaError_t radix_sort_u32_wide(uint32_t* keys, uint32_t* keys_alt, uint64_t* vals, uint64_t* vals_alt,
                                const int64_t* d_n, int64_t n_max, int bits, void* temp, cudaStream_t s,
                                bool* in_alt);

}  // namespace ivfk
