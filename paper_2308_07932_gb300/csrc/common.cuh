// common.cuh - device-side types and helpers shared by the build and count
// kernels of the balanced butterfly path (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bb {

// counts kernel launches issued by the library (reported by bb_launch_count)
void note_launch();

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP = 32;

// device error word bits (set with atomicOr, read once per call)
enum : uint32_t {
    E_ROWPTR = 1u,      // rowptr not monotone / out of range
    E_COL = 2u,         // column id outside [0, nV)
    E_SIGN = 4u,        // sign not +1 / -1
    E_DUP = 8u,         // an edge listed twice
    E_PROBE = 16u,      // hash probe bound exceeded (must not happen)
    E_INTERNAL = 64u,   // an internal bound check failed
    E_WAIT = 128u,      // a bounded device-side wait gave up (reported as a timeout)
};

// Counter fields: per (anchor, endpoint) pair the symmetric-wedge count S in
// bits 0..15 and the asymmetric-wedge count A in bits 16..31. Both are at
// most the anchor's degree (the anchor is the pair's lower-priority vertex,
// Def. 4, so its degree is the smaller one), which fits 16 bits up to
// MAX_DEGREE; anchors of higher degree are counted with 32-bit fields
// (wide dense jobs).
constexpr uint32_t MAX_DEGREE = 65535;
constexpr uint32_t INC_SYM = 1u;
constexpr uint32_t INC_ASYM = 1u << 16;

// Rank-space CSR of one side (U = 0, V = 1). Rows are indexed by side rank
// (position of the vertex among its side in ascending degree priority,
// Def. 4); each row lists the neighbours' side ranks ascending, with the
// edge sign folded into bit 0 (1 = negative).
struct SideCSR {
    int64_t n;            // vertices on this side
    int64_t *off;         // [n+1] row offsets
    uint32_t *adj;        // [nE]  (neighbour side rank << 1) | negative
    uint4 *md;            // [nE]  per entry (w -> v), the wedges it starts, as absolute
                          //       positions in the other side's adj: x = first
                          //       neighbour of v ranked above both v and w, y = first of
                          //       those inside the hub window, z = end of v's row,
                          //       w = sign bit of the edge (w, v)
    uint32_t *id_of_sr;   // [n]   side rank -> input id
    uint32_t *sr_of_id;   // [n]   input id -> side rank
    uint32_t *grank;      // [n]   side rank -> global priority rank
    uint32_t *deg;        // [n]   side rank -> degree
    uint32_t *lo;         // [n]   scratch of the build (degree keys of the rank sort)
    uint64_t *work;       // [n]   side rank -> wedges anchored at this vertex
    uint64_t *work_nh;    // [n]   of those, wedges whose endpoint lies below the hub window
    unsigned long long *pv;  // [n] balanced butterflies containing each vertex (when asked)
};

__host__ __device__ __forceinline__ uint64_t c2(uint64_t n) {
    return n < 2 ? 0 : (n & 1 ? n * ((n - 1) >> 1) : (n >> 1) * (n - 1));
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// inclusive warp scan of 32-bit values
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= (unsigned)d) x += y;
    }
    return x;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
    return x;
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
    return x;
}

// first index i in [lo, hi) with a[i] >= key (a ascending)
__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *a, int64_t lo, int64_t hi,
                                                   uint32_t key) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void set_error(uint32_t *err, uint32_t bits) { atomicOr(err, bits); }

// Fibonacci hashing of an endpoint key into a table of 2^(32 - shift) slots
__device__ __forceinline__ uint32_t hash_slot(uint32_t key, uint32_t shift) {
    return (key * 0x9E3779B1u) >> shift;
}

}  // namespace bb
