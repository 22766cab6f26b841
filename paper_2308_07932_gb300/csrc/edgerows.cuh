// edgerows.cuh - the input row of every edge of a block's step of
// consecutive input edges, without a search per edge (used by the row fill
// of the build and by the per-edge output).
//
// Two warps find the step's first and last row (32 probes per round of a
// warp search over rowptr); every row of the step marks its first edge of
// the step in shared memory and a block-wide running maximum gives each
// edge its row, however many empty rows the step spans.
#pragma once
#include "common.cuh"

namespace bb {
namespace edgerows {

constexpr int THREADS = 256;    // threads of a block that calls step_rows
constexpr int EDGES = 2048;     // edges per step
constexpr int PER = EDGES / THREADS;

struct Smem {
    int64_t row_lim[2];
    uint32_t srow[EDGES];  // per edge of the step: its row - u0 + 1
    uint32_t wmax[THREADS / 32];
};

// last u in [lo, hi) with rp[u] <= e (rp[lo] <= e), by a whole warp (all
// lanes call it with the same arguments): each round probes 31 evenly
// spaced rows of (lo, hi) and keeps the gap between the last one at or
// below e and the next
__device__ __forceinline__ int64_t row_of_warp(const int64_t *rp, int64_t lo, int64_t hi,
                                               int64_t e, unsigned lane) {
    while (hi - lo > 1) {
        const int64_t p = lo + ((hi - lo) * (int64_t)(lane + 1)) / 32;
        const bool le = lane < 31 && rp[p] <= e;
        const int c = __popc(__ballot_sync(FULL, le));  // the true probes form a prefix
        const int64_t nlo = c > 0 ? __shfl_sync(FULL, p, c - 1) : lo;
        const int64_t nhi = c < 31 ? __shfl_sync(FULL, p, c) : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// block-wide inclusive running maximum of a[0..EDGES), PER consecutive
// values per thread
__device__ __forceinline__ void running_max(uint32_t *a, uint32_t *wmax) {
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    uint32_t v[PER], m = 0;
#pragma unroll
    for (int k = 0; k < PER; k++) {
        m = max(m, a[t * PER + k]);
        v[k] = m;
    }
    uint32_t x = m;  // inclusive warp scan (max) of the threads' maxima
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= (unsigned)d) x = max(x, y);
    }
    if (lane == 31) wmax[t >> 5] = x;
    __syncthreads();
    uint32_t before = __shfl_up_sync(FULL, x, 1);
    if (lane == 0) before = 0;
    for (int w = 0; w < (t >> 5); w++) before = max(before, wmax[w]);
#pragma unroll
    for (int k = 0; k < PER; k++) a[t * PER + k] = max(before, v[k]);
}

// The rows of the edges [e0, e1) (e1 - e0 <= EDGES) of a U-side CSR with
// nU rows: returns u0; edge e's row is u0 + sm.srow[e - e0] - 1. All
// THREADS threads of the block call it; sm is valid until the caller's
// next barrier-free reuse (callers sync before the next step).
__device__ __forceinline__ int64_t step_rows(const int64_t *rowptr, int64_t nU, int64_t e0,
                                             int64_t e1, Smem &sm) {
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    if (t < 64) {
        const int64_t u = row_of_warp(rowptr, 0, nU, t < 32 ? e0 : e1 - 1, lane);
        if (lane == 0) sm.row_lim[t >> 5] = u;
    }
    for (int i = t; i < EDGES; i += THREADS) sm.srow[i] = 0u;
    __syncthreads();
    const int64_t u0 = sm.row_lim[0], u1 = sm.row_lim[1];
    // each row marks its first edge in the step (rows with edges have
    // distinct starts; u0's is clamped to e0)
    for (int64_t u = u0 + t; u <= u1; u += THREADS) {
        const int64_t a = rowptr[u], b = rowptr[u + 1];
        const int64_t st = a > e0 ? a : e0;
        if (b > st && st < e1) sm.srow[st - e0] = (uint32_t)(u - u0 + 1);
    }
    __syncthreads();
    running_max(sm.srow, sm.wmax);
    __syncthreads();
    return u0;
}

}  // namespace edgerows
}  // namespace bb
