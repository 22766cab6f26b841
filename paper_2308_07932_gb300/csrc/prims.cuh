// prims.cuh - device-wide exclusive scan and stable LSD radix sort used by
// the graph build (vertex ranking). Written for this library; no external
// template library is used.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bb {

// Bytes of temporary storage scan_exclusive needs for n elements.
size_t scan_temp_bytes(int64_t n);

// out[i] = sum_{j<i} in[i]; out[n] = total. in/out may alias. T = uint32_t,
// uint64_t or int64_t (uint32 inputs scanned into int64 outputs use the
// widening overload).
void scan_exclusive_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n, void *temp,
                               cudaStream_t s);
void scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, void *temp,
                        cudaStream_t s);

// Stable sort of (key, value) pairs by the low `key_bits` bits of key.
size_t radix_temp_bytes(int64_t n);
// Sorts keys[0..n) / vals[0..n) in place (using the alternate buffers).
void radix_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                          int64_t n, int key_bits, void *temp, cudaStream_t s);

}  // namespace bb
