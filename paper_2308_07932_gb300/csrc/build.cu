// build.cu - from the input U-side CSR to the ranked, sign-packed CSR of
// both sides, the wedge-suffix starts, per-anchor work and work classes.
//
// Steps (paper: Algorithm 2 lines 2-3 "calculate p(u)" and "rearrange
// Gamma(u) in ascending order"; Def. 4 for the priority; the binning sort of
// the complexity analysis for ordering by degree):
//   1. validate the CSR and count degrees;
//   2. rank each side by (degree, id) and derive the global priority rank;
//   3. place every edge in the rows of both endpoints, keyed by the
//      neighbour's side rank with the sign in bit 0, and sort each row;
//   4. for every entry w -> v, the start of the suffix of v's row ranked
//      above both v and w, and the wedges anchored at each vertex;
//   5. split anchors into work classes ordered by decreasing work.
#include <algorithm>
#include <mutex>
#include "edgerows.cuh"
#include "graph.cuh"
#include "prims.cuh"

namespace bb {

namespace {

constexpr int BT = 256;  // default threads per block for simple kernels
constexpr uint32_t DEG_COPIES = 8;  // V degree counter replicas during validation

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------ 1. validate
// largest of the warp's values into *maxdeg (all lanes of the warp call it);
// the atomic only when the value exceeds the maximum seen so far (every
// warp's atomic on one address serialised: 45 us for 2M U vertices)
__device__ __forceinline__ void warp_max_to(uint32_t v, uint32_t *maxdeg) {
    v = __reduce_max_sync(FULL, v);
    if (lane_id() == 0 && v > *(volatile uint32_t *)maxdeg) atomicMax(maxdeg, v);
}

// rows: rowptr monotone within [0, nE]; U degrees (a degree fits 32 bits
// because nE < 2^32) and their maximum
__global__ void k_validate_rows(const int64_t *rowptr, int64_t nU, int64_t nE, uint32_t *degU,
                                uint32_t *err, uint32_t *maxdeg) {
    uint32_t mx = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nU;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = rowptr[u], b = rowptr[u + 1];
        uint32_t d = 0;
        if (a < 0 || b < a || b > nE) set_error(err, E_ROWPTR);
        else d = (uint32_t)(b - a);
        degU[u] = d;
        mx = d > mx ? d : mx;
        if (u == 0 && a != 0) set_error(err, E_ROWPTR);
        if (u == nU - 1 && b != nE) set_error(err, E_ROWPTR);
    }
    warp_max_to(mx, maxdeg);
}

// edges: column in range, sign +1/-1, and the V degrees. A hub's degree
// counter takes one atomic per edge; the counts go to one of `copies`
// replicas (by block, replica c at degc + c * stride) so that a hub's edges
// spread over several addresses, summed by k_max_degree.
__global__ void k_validate_edges(const int32_t *col, const int8_t *sign, int64_t nE, int64_t nV,
                                 uint32_t *degc, int64_t stride, uint32_t copies, uint32_t *err) {
    uint32_t *deg = degc + (int64_t)(blockIdx.x & (copies - 1u)) * stride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nE;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = col[e];
        int8_t sg = sign[e];
        if (c < 0 || (int64_t)c >= nV) set_error(err, E_COL);
        else atomicAdd(&deg[c], 1u);
        if (sg != 1 && sg != -1) set_error(err, E_SIGN);
    }
}

// V degrees as the sum of the replicas (written to deg) and their largest
__global__ void k_max_degree(const uint32_t *degc, int64_t stride, uint32_t copies, uint32_t *deg,
                             int64_t n, uint32_t *maxdeg) {
    uint32_t mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t d = 0;
        for (uint32_t c = 0; c < copies; c++) d += degc[c * stride + i];
        if (copies > 1) deg[i] = d;
        mx = d > mx ? d : mx;
    }
    warp_max_to(mx, maxdeg);
}

__global__ void k_iota(uint32_t *a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

// ------------------------------------------------------------- 2. ranking
// sorted_deg/sorted_id: a side's vertices in ascending (degree, id) order.
__global__ void k_side_rank(const uint32_t *sorted_id, const uint32_t *sorted_deg, int64_t n,
                            SideCSR S) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t id = sorted_id[r];
        S.id_of_sr[r] = id;
        S.sr_of_id[id] = (uint32_t)r;
        S.deg[r] = sorted_deg[r];
    }
}

// Global priority (Def. 4) over U and V with ids compared as gid = u for U
// and |U| + v for V: a U vertex of degree d outranks every V vertex of
// degree < d; a V vertex of degree d outranks every U vertex of degree <= d.
__global__ void k_global_rank(SideCSR S, const uint32_t *other_deg, int64_t n_other, int is_u) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < S.n;
         r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t d = S.deg[r];
        int64_t lo = 0, hi = n_other;
        if (is_u) {  // first other index with deg >= d
            while (lo < hi) { int64_t m = (lo + hi) >> 1; if (other_deg[m] < d) lo = m + 1; else hi = m; }
        } else {     // first other index with deg > d
            while (lo < hi) { int64_t m = (lo + hi) >> 1; if (other_deg[m] <= d) lo = m + 1; else hi = m; }
        }
        S.grank[r] = (uint32_t)(r + lo);
    }
}

// --------------------------------------------------------------- 3. rows
// Each input edge e is written into the rows of both endpoints: the U-side
// entry keeps the input position within its row u; the V-side entry takes
// a free slot of v's row. Each entry is written as one key (packed entry <<
// 32 | input edge id) for the row sorts. A block takes edgerows::EDGES
// consecutive edges per step and finds their rows without a search per
// edge (edgerows.cuh). The V rows of the step's edges are gathered in a
// shared hash, so that each distinct V row takes its slots with one global
// atomic per step (hub rows take edges from most steps).
constexpr int FILL_THREADS = edgerows::THREADS;
constexpr int FILL_EDGES = edgerows::EDGES;
constexpr int FILL_PER = edgerows::PER;
constexpr uint32_t FILL_SLOTS = 4096;
constexpr uint32_t FILL_EMPTY = 0xffffffffu;
constexpr uint32_t FILL_HASH_BITS = 12;
static_assert(FILL_SLOTS == 1u << FILL_HASH_BITS && FILL_SLOTS >= 2 * FILL_EDGES, "fill hash");

__global__ void __launch_bounds__(FILL_THREADS) k_fill(
    const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
    const int8_t *__restrict__ sign, int64_t nU, int64_t nE, SideCSR U, SideCSR V,
    uint32_t *cursorV, uint32_t *keyU, uint32_t *keyV, uint32_t *err) {
    __shared__ edgerows::Smem er;
    __shared__ uint32_t hkey[FILL_SLOTS], hcnt[FILL_SLOTS];
    const int t = threadIdx.x;
    const uint32_t *srow = er.srow;
    for (uint32_t i = t; i < FILL_SLOTS; i += FILL_THREADS) {
        hkey[i] = FILL_EMPTY;
        hcnt[i] = 0u;
    }
    for (int64_t e0 = blockIdx.x * (int64_t)FILL_EDGES; e0 < nE;
         e0 += (int64_t)gridDim.x * FILL_EDGES) {
        const int64_t e1 = nE - e0 > FILL_EDGES ? e0 + FILL_EDGES : nE;
        const int64_t u0 = edgerows::step_rows(rowptr, nU, e0, e1, er);
        // 1. U entries; V rows into the shared hash, with each edge's rank
        // among the step's edges of its row (the loads of all the thread's
        // edges are issued before the hash inserts)
        uint32_t slot[FILL_PER], loc[FILL_PER], rvk[FILL_PER], kv[FILL_PER];
#pragma unroll
        for (int k = 0; k < FILL_PER; k++) {
            const int64_t e = e0 + k * FILL_THREADS + t;
            slot[k] = FILL_SLOTS;
            loc[k] = rvk[k] = kv[k] = 0u;
            if (e >= e1) continue;
            const int64_t u = u0 + srow[e - e0] - 1;
            const int64_t ru = rowptr[u];
            const uint32_t r = U.sr_of_id[u];
            const uint32_t neg = sign[e] < 0 ? 1u : 0u;
            const uint32_t rv = V.sr_of_id[(uint32_t)col[e]];
            keyU[U.off[r] + (e - ru)] = (rv << 1) | neg;
            slot[k] = 0u;
            rvk[k] = rv;
            kv[k] = (r << 1) | neg;
        }
#pragma unroll
        for (int k = 0; k < FILL_PER; k++) {
            if (slot[k] == FILL_SLOTS) continue;
            const uint32_t rv = rvk[k];
            uint32_t h = hash_slot(rv + 1u, 32 - FILL_HASH_BITS);
            uint32_t probe = 0;
            for (; probe < FILL_SLOTS; probe++) {
                const uint32_t cur = *((volatile uint32_t *)&hkey[h]);
                if (cur == rv) break;
                if (cur == FILL_EMPTY) {
                    const uint32_t old = atomicCAS(&hkey[h], FILL_EMPTY, rv);
                    if (old == FILL_EMPTY || old == rv) break;
                }
                h = (h + 1) & (FILL_SLOTS - 1);
            }
            if (probe == FILL_SLOTS) {  // cannot happen at load <= 1/2
                set_error(err, E_INTERNAL);
                slot[k] = FILL_SLOTS;
                continue;
            }
            slot[k] = h;
            loc[k] = atomicAdd(&hcnt[h], 1u);
        }
        __syncthreads();
        // 2. one global atomic per distinct V row of the step: the base of
        // its slots replaces its count
        for (uint32_t i = t; i < FILL_SLOTS; i += FILL_THREADS) {
            const uint32_t c = hcnt[i];
            if (!c) continue;
            hcnt[i] = atomicAdd(&cursorV[hkey[i]], c);
            hkey[i] = FILL_EMPTY;
        }
        __syncthreads();
        // 3. V entries
#pragma unroll
        for (int k = 0; k < FILL_PER; k++) {
            if (slot[k] == FILL_SLOTS) continue;
            const int64_t e = e0 + k * FILL_THREADS + t;
            const int64_t pv = V.off[rvk[k]] + hcnt[slot[k]] + loc[k];
            keyV[pv] = kv[k];
        }
        __syncthreads();
        for (uint32_t i = t; i < FILL_SLOTS; i += FILL_THREADS) hcnt[i] = 0u;
        // (the next step's first barrier orders these stores before its use)
    }
}

// Row length classes of a side (rows are in ascending degree, so each class
// is a contiguous range of side ranks): bounds[k] = first side rank whose
// degree exceeds ROW_LIMS[k]; bounds[NLIMS] = n.
constexpr int NLIMS = 12;
__constant__ uint32_t ROW_LIMS[NLIMS] = {1u,  2u,   4u,   8u,    16u,   32u,
                                         64u, 128u, 256u, 512u, 2048u, 16384u};
constexpr int LIM_LONG = 10;  // class of the rows above 2,048 entries

__global__ void k_row_bounds(const uint32_t *deg, int64_t n, int64_t *bounds) {
    int k = threadIdx.x;
    if (k == NLIMS) bounds[NLIMS] = n;
    if (k >= NLIMS) return;
    uint32_t lim = ROW_LIMS[k];
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t m = (lo + hi) >> 1; if (deg[m] <= lim) lo = m + 1; else hi = m; }
    bounds[k] = lo;
}


// A row key is the entry itself (neighbour side rank << 1 | negative); a
// row's ranks are distinct, so equal ranks next to each other after a sort
// are a duplicate edge.
__device__ __forceinline__ bool same_rank(uint32_t a, uint32_t b) { return (a >> 1) == (b >> 1); }

// rows of degree 0 or 1: nothing to sort, unpack the key
__global__ void k_rows_single(SideCSR S, const uint32_t *keys, const int64_t *bounds) {
    const int64_t r1 = bounds[0];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < r1;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = S.off[r];
        if (S.off[r + 1] > b) S.adj[b] = keys[b];
    }
}

// rows of (WIDTH/2, WIDTH] entries, WIDTH <= 32: 32/WIDTH rows per warp,
// bitonic sort in registers across WIDTH lanes
template <int WIDTH>
__global__ void k_sort_rows_sub(SideCSR S, const uint32_t *keys, const int64_t *bounds, int lo_k,
                                uint32_t *err) {
    constexpr int PER = 32 / WIDTH;
    const int64_t r0 = bounds[lo_k], r1 = bounds[lo_k + 1];
    const unsigned lane = lane_id();
    const uint32_t el = lane % WIDTH;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t rb = r0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * PER; rb < r1;
         rb += warps * PER) {
        const int64_t r = rb + lane / WIDTH;
        int64_t b = 0;
        uint32_t d = 0;
        if (r < r1) {
            b = S.off[r];
            d = (uint32_t)(S.off[r + 1] - b);
        }
        uint32_t x = el < d ? keys[b + el] : ~0u;
#pragma unroll
        for (int k = 2; k <= WIDTH; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint32_t y = __shfl_xor_sync(FULL, x, j);
                const bool keep_min = ((el & j) == 0) == ((el & k) == 0);
                x = keep_min ? min(x, y) : max(x, y);
            }
        }
        const uint32_t prev = __shfl_up_sync(FULL, x, 1);
        if (el < d) {
            S.adj[b + el] = x;
            if (el > 0 && same_rank(prev, x)) set_error(err, E_DUP);
        }
    }
}

// rows of (16 K, 32 K] entries (K = 2 to 16: 33 to 512 entries): one warp
// per row, bitonic sort in registers with K entries per lane (entry i in
// lane i / K, slot i % K): the partner at distance j < K is in the lane's
// own registers, a farther one a shuffle away. (A shared-memory bitonic sort
// of these rows took about 2.5 times the instructions.)
template <int K>
__global__ void __launch_bounds__(256) k_sort_rows_warpreg(SideCSR S, const uint32_t *keys,
                                                           const int64_t *bounds, int lo_k,
                                                           uint32_t *err) {
    constexpr uint32_t P = 32 * K;
    const int64_t r0 = bounds[lo_k], r1 = bounds[lo_k + 1];
    const unsigned lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = r0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); r < r1;
         r += warps) {
        const int64_t b = S.off[r];
        const uint32_t d = (uint32_t)(S.off[r + 1] - b);
        uint32_t x[K];
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint32_t i = lane * K + q;
            x[q] = i < d ? keys[b + i] : ~0u;
        }
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j >= (uint32_t)K; j >>= 1) {  // partners in other lanes
#pragma unroll
                for (int q = 0; q < K; q++) {
                    const uint32_t i = lane * K + q;
                    const uint32_t y = __shfl_xor_sync(FULL, x[q], j / K);
                    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                    x[q] = keep_min ? min(x[q], y) : max(x[q], y);
                }
            }
#pragma unroll
            for (int j = K / 2; j > 0; j >>= 1) {  // partners in the lane's registers
                if ((uint32_t)j >= k) continue;
#pragma unroll
                for (int q = 0; q < K; q++) {
                    if (q & j) continue;  // q is the lower entry of the pair (q, q | j)
                    const bool asc = ((lane * K + q) & k) == 0;
                    const uint32_t a = x[q], c = x[q | j];
                    const bool swap = asc ? a > c : a < c;
                    x[q] = swap ? c : a;
                    x[q | j] = swap ? a : c;
                }
            }
        }
        // write back; a repeated rank is a duplicate edge
        const uint32_t prev_last = __shfl_up_sync(FULL, x[K - 1], 1);
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint32_t i = lane * K + q;
            if (i < d) {
                S.adj[b + i] = x[q];
                const uint32_t pv = q ? x[q - 1] : prev_last;
                if (i > 0 && same_rank(pv, x[q])) set_error(err, E_DUP);
            }
        }
    }
}

// rows of (512, CAP] entries: one CTA per row, bitonic sort in shared memory
template <int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) k_sort_rows_smem(SideCSR S, const uint32_t *keys,
                                                            const int64_t *bounds, int lo_k,
                                                            uint32_t *err) {
    extern __shared__ uint32_t sbuf[];
    const int64_t r0 = bounds[lo_k], r1 = bounds[lo_k + 1];
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        int64_t b = S.off[r];
        uint32_t d = (uint32_t)(S.off[r + 1] - b);
        uint32_t P = 1;
        while (P < d) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += THREADS)
            sbuf[i] = i < d ? keys[b + i] : ~0u;
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                // compare-exchange pairs (i, i + j), i with bit j clear: P/2 of them
                for (uint32_t q = threadIdx.x; q < P / 2; q += THREADS) {
                    const uint32_t i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                    const uint32_t a = sbuf[i], c = sbuf[i | j];
                    if ((a > c) == ((i & k) == 0)) { sbuf[i] = c; sbuf[i | j] = a; }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < d; i += THREADS) {
            const uint32_t x = sbuf[i];
            S.adj[b + i] = x;
            if (i > 0 && same_rank(sbuf[i - 1], x)) set_error(err, E_DUP);
        }
        __syncthreads();
    }
}

// rows of more than 2048 entries: one CTA per row, stable LSD radix sort
// (8-bit digits) through two global buffers
constexpr int RR_THREADS = 1024;
constexpr int RR_WARPS = RR_THREADS / 32;

__global__ void __launch_bounds__(RR_THREADS) k_sort_rows_radix(SideCSR S, uint32_t *keys,
                                                                uint32_t *alt,
                                                                const int64_t *bounds, int lo_k,
                                                                int hi_k, int key_bits,
                                                                uint32_t *err) {
    __shared__ uint32_t wcnt[RR_WARPS][256];
    __shared__ uint32_t run[256];
    const int64_t r0 = bounds[lo_k], r1 = bounds[hi_k];
    const int t = threadIdx.x, warp = t >> 5;
    const unsigned lane = lane_id();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int passes = (key_bits + 7) / 8;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        int64_t b = S.off[r];
        int64_t d = S.off[r + 1] - b;
        uint32_t *A = keys + b, *B = alt + b;
        for (int k = t; k < RR_WARPS * 256; k += RR_THREADS) (&wcnt[0][0])[k] = 0;
        __syncthreads();
        uint32_t *src = A, *dst = B;
        for (int p = 0; p < passes; p++) {
            const int shift = 8 * p;
            if (t < 256) run[t] = 0;
            __syncthreads();
            for (int64_t i = t; i < d; i += RR_THREADS) atomicAdd(&run[(src[i] >> shift) & 255u], 1u);
            __syncthreads();
            if (t < 32) {  // exclusive scan of 256 bins by one warp (8 per lane)
                uint32_t v[8], s = 0;
#pragma unroll
                for (int k = 0; k < 8; k++) { v[k] = run[t * 8 + k]; s += v[k]; }
                uint32_t incl = warp_incl_scan(s);
                uint32_t acc = incl - s;
#pragma unroll
                for (int k = 0; k < 8; k++) { run[t * 8 + k] = acc; acc += v[k]; }
            }
            __syncthreads();
            for (int64_t base = 0; base < d; base += RR_THREADS) {
                int64_t i = base + t;
                bool valid = i < d;
                uint32_t x = valid ? src[i] : 0u;
                uint32_t dg = valid ? (uint32_t)((x >> shift) & 255u) : 256u + lane;
                unsigned peers = __match_any_sync(FULL, dg);
                uint32_t rank = __popc(peers & lt_mask);
                if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
                __syncthreads();
                if (t < 256) {
                    uint32_t s = run[t];
                    for (int w = 0; w < RR_WARPS; w++) { uint32_t c = wcnt[w][t]; wcnt[w][t] = s; s += c; }
                    run[t] = s;
                }
                __syncthreads();
                if (valid) dst[wcnt[warp][dg] + rank] = x;
                __syncthreads();
                if (t < 256)
                    for (int w = 0; w < RR_WARPS; w++) wcnt[w][t] = 0;
                __syncthreads();
            }
            uint32_t *tmp = src; src = dst; dst = tmp;
        }
        for (int64_t i = t; i < d; i += RR_THREADS) {
            const uint32_t x = src[i];
            S.adj[b + i] = x;
            if (i > 0 && same_rank(src[i - 1], x)) set_error(err, E_DUP);
        }
        __syncthreads();
    }
}

// Rows of more than 2048 entries, when the other side is at most
// BM_MAX_SLICES * BM_RANKS vertices: one CTA per row. The neighbour ranks of
// a row are distinct (a repeated one is a duplicate edge), so a bitmap over
// the rank range sorts them: each entry sets its rank's bit, a block-wide
// exclusive scan of the words' popcounts gives each word's first position,
// and an entry's position is that plus the set bits below its own. The
// rank range is covered in slices of BM_RANKS ranks (the bitmap and the
// prefixes of one slice fill 128 KiB of shared memory), one pass over the
// row per slice. Work per row: its entries times the slices, plus the
// other side's vertices / 32 words per slice.
constexpr int BM_THREADS = 1024;
constexpr uint32_t BM_WORDS = 16384;
constexpr uint32_t BM_RANKS = BM_WORDS * 32;
constexpr uint32_t BM_MAX_SLICES = 8;
constexpr uint32_t BM_PER = BM_WORDS / BM_THREADS;  // words per thread in the scan
constexpr size_t BM_SMEM = 2 * BM_WORDS * 4;

__global__ void __launch_bounds__(BM_THREADS) k_sort_rows_bitmap(SideCSR S, const uint32_t *keys,
                                                                 const int64_t *bounds, int lo_k,
                                                                 int hi_k, uint32_t n_other,
                                                                 uint32_t *err) {
    extern __shared__ uint32_t bm_raw[];
    uint32_t *bm = bm_raw, *pre = bm_raw + BM_WORDS;
    __shared__ uint32_t wtot[BM_THREADS / 32];
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    const int64_t r0 = bounds[lo_k], r1 = bounds[hi_k];
    const uint32_t slices = (n_other + BM_RANKS - 1) / BM_RANKS;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const int64_t b = S.off[r];
        const uint32_t d = (uint32_t)(S.off[r + 1] - b);
        uint32_t placed = 0;  // entries of the earlier slices
        for (uint32_t sl = 0; sl < slices; sl++) {
            const uint32_t lo = sl * BM_RANKS;
            const uint32_t span = n_other - lo < BM_RANKS ? n_other - lo : BM_RANKS;
            for (uint32_t i = t; i < BM_WORDS; i += BM_THREADS) bm[i] = 0u;
            __syncthreads();
            for (uint32_t i = t; i < d; i += BM_THREADS) {
                const uint32_t rr = (keys[b + i] >> 1) - lo;
                if (rr < span) {
                    const uint32_t bit = 1u << (rr & 31u);
                    if (atomicOr(&bm[rr >> 5], bit) & bit) set_error(err, E_DUP);
                }
            }
            __syncthreads();
            // exclusive prefix of the words' popcounts: BM_PER words a thread
            uint32_t c[BM_PER], sum = 0;
#pragma unroll
            for (uint32_t k = 0; k < BM_PER; k++) {
                c[k] = __popc(bm[t * BM_PER + k]);
                sum += c[k];
            }
            const uint32_t incl = warp_incl_scan(sum);
            if (lane == 31) wtot[t >> 5] = incl;
            __syncthreads();
            uint32_t ex = incl - sum, total = 0;
            for (int w = 0; w < BM_THREADS / 32; w++) {
                const uint32_t v = wtot[w];
                if (w < (t >> 5)) ex += v;
                total += v;
            }
#pragma unroll
            for (uint32_t k = 0; k < BM_PER; k++) {
                pre[t * BM_PER + k] = ex;
                ex += c[k];
            }
            __syncthreads();
            for (uint32_t i = t; i < d; i += BM_THREADS) {
                const uint32_t x = keys[b + i];
                const uint32_t rr = (x >> 1) - lo;
                if (rr < span) {
                    const uint32_t w = rr >> 5;
                    const uint32_t pos =
                        placed + pre[w] + __popc(bm[w] & ((1u << (rr & 31u)) - 1u));
                    if (pos < d) S.adj[b + pos] = x;
                }
            }
            placed += total;
            __syncthreads();  // the next slice rewrites the bitmap
        }
        if (placed != d && t == 0) set_error(err, E_DUP);  // only repeated ranks leave gaps
    }
}

// per device, once (any thread may build on any device): SM count and the
// shared-memory opt-in of the bitmap row sort
constexpr int BUILD_MAX_DEVICES = 64;
int g_build_sms[BUILD_MAX_DEVICES];
std::once_flag g_build_once[BUILD_MAX_DEVICES];

int build_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= BUILD_MAX_DEVICES) {
        cudaGetLastError();
        dev = 0;
    }
    std::call_once(g_build_once[dev], [dev]() {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, dev);
        g_build_sms[dev] = prop.multiProcessorCount;
        cudaFuncSetAttribute(k_sort_rows_bitmap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BM_SMEM);
    });
    return g_build_sms[dev] > 0 ? g_build_sms[dev] : 1;
}

// Per row of a side: the row vertex's global rank, and as absolute
// positions in the side's adjacency the row's end, lo (the first neighbour
// of higher global priority than the row's vertex; the neighbours below it
// form a prefix) and the first neighbour inside the other side's hub window
// (side ranks >= window_base). One 16-byte record per row, read once per
// entry by k_md_work.
__global__ void k_row_info(SideCSR S, SideCSR O, uint32_t window_base, uint4 *info) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < S.n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = S.off[r], e = S.off[r + 1];
        const uint32_t g = S.grank[r];
        int64_t lo = b, hi = e;
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (O.grank[S.adj[m] >> 1] < g) lo = m + 1; else hi = m;
        }
        const int64_t h = lower_bound_u32(S.adj, b, e, window_base << 1);
        info[r] = make_uint4(g, (uint32_t)e, (uint32_t)lo, (uint32_t)h);
    }
}

// ------------------------------------------------- 4. suffixes and work
// For the entry w -> v at position p of anchor w's row: the wedge suffix of
// v's row holds the neighbours ranked above max(v, w). If v outranks w that
// is v's own upper part, from lo(v); otherwise w lies in that upper part
// and the suffix starts right after w's position there (w and the suffix
// are on the same side), found by binary search. A block takes
// edgerows::EDGES consecutive entries per step and finds their rows from
// the side's offsets (edgerows.cuh). The per-row sums of suffix lengths
// (wedges) and of their parts below the hub window are reduced per warp
// segment, then added per row.
__global__ void __launch_bounds__(edgerows::THREADS) k_md_work(SideCSR S, SideCSR O,
                                                               const uint4 *__restrict__ info_o,
                                                               int64_t nE,
                                                               unsigned long long *wedges,
                                                               uint32_t *err) {
    __shared__ edgerows::Smem er;
    __shared__ unsigned long long block_sum;
    const int t = threadIdx.x;
    const unsigned lane = lane_id();
    if (t == 0) block_sum = 0;
    unsigned long long mine = 0;
    for (int64_t p0 = blockIdx.x * (int64_t)edgerows::EDGES; p0 < nE;
         p0 += (int64_t)gridDim.x * edgerows::EDGES) {
        const int64_t p1 = nE - p0 > edgerows::EDGES ? p0 + edgerows::EDGES : nE;
        const int64_t r0 = edgerows::step_rows(S.off, S.n, p0, p1, er);
        // all lanes of a warp run every iteration (shuffles below)
#pragma unroll 1
        for (int k = 0; k < edgerows::PER; k++) {
            const int64_t p = p0 + k * edgerows::THREADS + t;
            const bool valid = p < p1;
            uint32_t r = 0xffffffffu, len = 0, nh = 0;
            if (valid) {
                r = (uint32_t)(r0 + er.srow[p - p0] - 1);
                const uint32_t ent = S.adj[p];
                const uint32_t v = ent >> 1;
                const uint4 vi = info_o[v];  // v's row: global rank, end, lo, hub start
                uint32_t st = vi.z;
                if (S.grank[r] > vi.x) {  // w outranks v: w is in v's upper part
                    const int64_t pw = lower_bound_u32(O.adj, vi.z, vi.y, r << 1);
                    if (pw >= vi.y || (O.adj[pw] >> 1) != r) set_error(err, E_INTERNAL);
                    st = (uint32_t)pw + 1u;
                }
                const uint32_t hs = vi.w > st ? vi.w : st;
                S.md[p] = make_uint4(st, hs, vi.y, ent & 1u);
                len = vi.y - st;
                nh = hs - st;
            }
            // segmented sums over runs of equal r within the warp
            const uint32_t rprev = __shfl_up_sync(FULL, r, 1);
            const bool head = lane == 0 || rprev != r;
            const unsigned heads = __ballot_sync(FULL, head);
            uint32_t a = len, b = nh;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t ya = __shfl_up_sync(FULL, a, d), yb = __shfl_up_sync(FULL, b, d);
                if (lane >= (unsigned)d) { a += ya; b += yb; }
            }
            const unsigned below = heads & ((2u << lane) - 1u);  // heads at or before me
            const int sstart = 31 - __clz(below);                 // my segment's head
            const uint32_t pa = __shfl_sync(FULL, a, sstart > 0 ? sstart - 1 : 0);
            const uint32_t pb = __shfl_sync(FULL, b, sstart > 0 ? sstart - 1 : 0);
            const uint32_t seg_a = a - (sstart > 0 ? pa : 0u), seg_b = b - (sstart > 0 ? pb : 0u);
            const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
            if (valid && tail) {
                if (seg_a) atomicAdd((unsigned long long *)&S.work[r], (unsigned long long)seg_a);
                if (seg_b) atomicAdd((unsigned long long *)&S.work_nh[r], (unsigned long long)seg_b);
            }
            mine += len;
        }
        __syncthreads();  // the next step rewrites the shared rows
    }
    mine = warp_sum_u64(mine);
    if (lane == 0 && mine) atomicAdd(&block_sum, mine);
    __syncthreads();
    if (t == 0 && block_sum) atomicAdd(wedges, block_sum);
}

// ------------------------------------------------------ 5. classification
constexpr int NB = 64;  // log2 work buckets

struct ClassifyTemp {
    uint32_t *meta;         // per anchor: 1 | cls << 1 | bucket << 3 | parts << 9 | wide << 31
                            // (0 = no work)
    uint32_t *grp;          // per anchor: split group id
    uint32_t *bucket_cnt;   // [NCLS][NB]
    uint32_t *bucket_base;  // [NCLS][NB]
};

constexpr uint64_t MIDDLE_COST = 8;
__device__ __forceinline__ uint32_t bucket_of(uint64_t w) { return 63u - (uint32_t)__clzll((long long)w); }

// decides each anchor's class (and split) and counts entries per bucket
__global__ void k_classify(SideCSR S, int side, ClassifyTemp T, DevGraph G) {
    __shared__ uint32_t cnt[NCLS * NB];
    __shared__ unsigned long long stats[3 * NCLS];
    for (int k = threadIdx.x; k < NCLS * NB; k += blockDim.x) cnt[k] = 0;
    if (threadIdx.x < 3 * NCLS) stats[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long my_w[NCLS] = {}, my_m[NCLS] = {};
    uint32_t my_a[NCLS] = {};
    // warp-uniform trip counts (the bucket counts are aggregated per warp)
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < S.n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = base + threadIdx.x;
        const bool in = r < S.n;
        uint64_t W = in ? S.work[r] : 0;
        uint32_t meta = 0, key = 0xffffffffu, nparts = 0;
        if (W > 0) {
            const uint64_t above = (uint64_t)(S.n - r - 1);
            const uint64_t wb = S.n > (int64_t)HUB_WINDOW ? (uint64_t)S.n - HUB_WINDOW : 0;
            const uint64_t above_nh = wb > (uint64_t)r + 1 ? wb - (uint64_t)r - 1 : 0;
            const uint64_t wnh = S.work_nh[r];
            const uint64_t dnh = wnh < above_nh ? wnh : above_nh;
            const uint64_t dh = W < above ? W : above;
            const uint32_t deg = (uint32_t)(S.off[r + 1] - S.off[r]);
            // an anchor of degree above MAX_DEGREE needs 32-bit tally fields:
            // a wide dense job; every other class packs them in 16 bits. The
            // hash classes also keep their wedge prefixes below 2^31.
            const bool wide = deg > MAX_DEGREE;
            uint32_t cls;
            const ClassifyParams &P = G.cls;
            if (wide) cls = CLS_DENSE;
            else if (deg <= WARP_DEG_MAX && W <= P.warp_w_max &&
                (W <= P.warp_small_w ? dh * 5 / 4 < WARP_CAP : dnh * 5 / 4 < WARP_CAP))
                cls = CLS_WARP;
            else if (W <= P.team_w_max && deg <= TEAM_DEG_MAX && dnh * 5 / 4 < TEAM_CAP)
                cls = CLS_TEAM;
            else if (above <= DENSE_CAP) cls = CLS_DENSE;
            else if (dnh * 2 < CTAH_CAP && wnh < (1ull << 31)) cls = CLS_CTAH;
            else cls = CLS_DENSE;  // endpoint range walked in DENSE_CAP windows
            uint32_t parts = 1;
            if (cls == CLS_DENSE && !wide && above <= DENSE_CAP && above > 0) {
                const uint64_t su = P.split_wedges;
                uint64_t unit = su > 4 * above ? su : 4 * above;
                uint64_t k = W / unit;
                uint32_t deg = (uint32_t)(S.off[r + 1] - S.off[r]);
                if (k > MAX_PARTS) k = MAX_PARTS;
                if (k > deg) k = deg;
                if (k >= 2) {
                    uint32_t jobs = atomicAdd(&G.ctr[CTR_SPLITJOBS], (uint32_t)k);
                    uint32_t goff = atomicAdd(&G.ctr[CTR_GPART], (uint32_t)above);
                    if (jobs + k <= MAX_SPLIT_JOBS && (uint64_t)goff + above <= G.gpart_cap) {
                        uint32_t gid = atomicAdd(&G.ctr[CTR_GROUPS], 1u);
                        G.groups[gid] = SplitGroup{(uint32_t)k, goff, (uint32_t)above, 0u};
                        T.grp[r] = gid;
                        parts = (uint32_t)k;
                    }
                }
            }
            // order of work within a class: wedges plus a middle's fixed cost
            // (its descriptor and chunk-scan slot, about MIDDLE_COST wedges),
            // so that anchors of many middles and few wedges start early
            const uint64_t est = W + MIDDLE_COST * (uint64_t)deg;
            uint32_t b = bucket_of(parts > 1 ? est / parts : est);
            meta = 1u | cls << 1 | b << 3 | parts << 9 | (wide ? 1u << 31 : 0u);
            key = cls * NB + b;
            nparts = parts;
            my_w[cls] += W;
            my_m[cls] += (unsigned long long)(S.off[r + 1] - S.off[r]);
            my_a[cls] += 1;
        }
        if (in) T.meta[r] = meta;
        // one shared atomic per distinct bucket in the warp
        const unsigned peers = __match_any_sync(FULL, key);
        const uint32_t total = __reduce_add_sync(peers, nparts);
        if (key != 0xffffffffu && (peers & ((1u << lane_id()) - 1u)) == 0)
            atomicAdd(&cnt[key], total);
    }
    // per-class work: summed per thread, then per warp, then one shared atomic
    // per warp (all threads updating the same few counters serialises)
#pragma unroll
    for (int c = 0; c < NCLS; c++) {
        const unsigned long long w = warp_sum_u64(my_w[c]), m = warp_sum_u64(my_m[c]);
        const uint32_t a = __reduce_add_sync(FULL, my_a[c]);
        if (lane_id() == 0) {
            if (w) atomicAdd(&stats[c], w);
            if (m) atomicAdd(&stats[NCLS + c], m);
            if (a) atomicAdd(&stats[2 * NCLS + c], (unsigned long long)a);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NCLS * NB; k += blockDim.x)
        if (cnt[k]) atomicAdd(&T.bucket_cnt[k], cnt[k]);
    if (threadIdx.x < 3 * NCLS && stats[threadIdx.x])
        atomicAdd(&G.cls_stats[threadIdx.x], stats[threadIdx.x]);
}

// bucket bases in decreasing bucket order; class totals to the counters
__global__ void k_bucket_base(ClassifyTemp T, DevGraph G) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int c = 0; c < NCLS; c++) {
        uint32_t acc = 0;
        for (int b = NB - 1; b >= 0; b--) {
            T.bucket_base[c * NB + b] = acc;
            acc += T.bucket_cnt[c * NB + b];
        }
        G.ctr[c] = acc;  // CTR_WARP, CTR_TEAM, CTR_CTAH, CTR_DENSE
    }
}

__global__ void k_emit(SideCSR S, int side, ClassifyTemp T, DevGraph G) {
    __shared__ uint32_t cnt[NCLS * NB];
    __shared__ uint32_t base[NCLS * NB];
    for (int k = threadIdx.x; k < NCLS * NB; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    // one pass per block-chunk so each block reserves its ranges once
    const int64_t chunk = blockDim.x;
    for (int64_t r0 = blockIdx.x * chunk; r0 < S.n; r0 += (int64_t)gridDim.x * chunk) {
        int64_t r = r0 + threadIdx.x;
        uint32_t meta = r < S.n ? T.meta[r] : 0u;
        uint32_t local = 0, key = 0, parts = 0;
        if (meta) {
            uint32_t cls = (meta >> 1) & 3u, b = (meta >> 3) & 63u;
            parts = (meta >> 9) & 0xffu;
            key = cls * NB + b;
            local = atomicAdd(&cnt[key], parts);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < NCLS * NB; k += blockDim.x) {
            if (cnt[k]) base[k] = T.bucket_base[k] + atomicAdd(&T.bucket_cnt[k], cnt[k]);
        }
        __syncthreads();
        if (meta) {
            uint32_t cls = key / NB;
            uint32_t pos = base[key] + local;
            uint32_t anchor = (uint32_t)r << 1 | (uint32_t)side;
            const uint32_t deg = (uint32_t)(S.off[r + 1] - S.off[r]);
            if (cls != CLS_DENSE) {
                const uint64_t W = S.work[r], wnh = S.work_nh[r];
                AnchorRec rec;
                rec.anchor = anchor;
                rec.rb = (uint32_t)S.off[r];
                rec.deg = deg;
                rec.W = W > 0xffffffffull ? 0xffffffffu : (uint32_t)W;
                rec.wnh = wnh > 0xffffffffull ? 0xffffffffu : (uint32_t)wnh;
                rec.flags = cls == CLS_WARP && W <= G.cls.warp_small_w ? REC_HASH_ALL : 0u;
                rec.pad1 = rec.pad2 = 0;
                AnchorRec *list = cls == CLS_WARP ? G.warp_list
                                  : cls == CLS_TEAM ? G.team_list : G.ctah_list;
                list[pos] = rec;
            } else {
                uint32_t grp = (meta >> 31) ? WIDE_JOB : parts > 1 ? T.grp[r] : NO_GROUP;
                for (uint32_t i = 0; i < parts; i++) {
                    uint32_t m0 = (uint32_t)((uint64_t)deg * i / parts);
                    uint32_t m1 = (uint32_t)((uint64_t)deg * (i + 1) / parts);
                    G.dense_jobs[pos + i] = DenseJob{anchor, m0, m1, grp};
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < NCLS * NB; k += blockDim.x) cnt[k] = 0;
        __syncthreads();
    }
}

struct Carver {
    char *p;
    template <typename T>
    T *take(size_t count) {
        T *r = (T *)p;
        p += align256(count * sizeof(T));
        return r;
    }
};

size_t side_bytes(int64_t n, int64_t nE) {
    return align256((size_t)(n + 1) * 8) + align256((size_t)nE * 4) + align256((size_t)nE * 16) +
           5 * align256((size_t)(n > 0 ? n : 1) * 4) + 3 * align256((size_t)(n > 0 ? n : 1) * 8);
}

}  // namespace

ProductPlan product_plan(int64_t nU, int64_t nV, int64_t nE) {
    ProductPlan p;
    const int side = nV < nU ? 1 : 0;
    const int64_t a = side ? nV : nU, b = side ? nU : nV;
    if (a < 2 || a > (int64_t)PROD_A_MAX || b >= (int64_t)PROD_B_MAX || nE < PROD_MIN_EDGES ||
        nE * PROD_DENSITY < a * b)
        return p;
    const uint64_t ap = ((uint64_t)a + 15) & ~15ull;
    const uint64_t tiles = ((ap + 127) / 128) * ((ap + 127) / 128);
    uint64_t split = 1;
    while (split * 2 * tiles <= PROD_TARGET_TILES && (uint64_t)b >= split * 2 * PROD_MIN_SLICE)
        split *= 2;
    const uint64_t kc = (((uint64_t)b + split - 1) / split + 63) & ~63ull;
    const uint64_t ld = split * kc;
    if (ap * ld > PROD_MAX_CELLS) return p;
    p.side = side;
    p.a = (uint32_t)a;
    p.b = (uint32_t)b;
    p.ap = (uint32_t)ap;
    p.split = (uint32_t)split;
    p.kc = (uint32_t)kc;
    p.ld = (uint32_t)ld;
    p.x_bytes = align256(2 * (size_t)ap * ld * 2);
    p.c_bytes = align256(2 * split * (size_t)ap * (size_t)ap * 4);
    p.cnt_bytes = align256(((size_t)a + (size_t)b + 2 * (size_t)ap + 2 * (size_t)ld) * 4);
    p.ws_bytes = (size_t)32 << 20;
    p.total = p.x_bytes + p.c_bytes + p.cnt_bytes + p.ws_bytes;
    return p;
}

BuildSizes build_sizes(int64_t nU, int64_t nV, int64_t nE, bool product) {
    int64_t n = nU + nV;
    int64_t nmax = std::max<int64_t>(std::max(nU, nV), 1);
    size_t g = side_bytes(nU, nE) + side_bytes(nV, nE);
    g += 3 * align256((size_t)(n + 1) * sizeof(AnchorRec));                  // warp/team/ctah lists
    g += align256((size_t)(n + MAX_SPLIT_JOBS) * sizeof(DenseJob));          // dense jobs
    g += align256((size_t)MAX_SPLIT_JOBS * sizeof(SplitGroup));              // groups
    g += align256((size_t)MAX_SPLIT_JOBS * 4);                               // gdone
    g += align256(gpart_entries(nE) * 4);
    g += align256(NCTR * 4) + 256 + 256 + 256 + align256(sizeof(CountScratch));
    size_t t = 0;
    t += align256((size_t)nU * 4 + 4) + align256((size_t)nV * 4 + 4);      // deg by id
    t += align256((size_t)nV * 4 + 4);                                       // cursor
    t += 3 * align256((size_t)nE * 4 + 4);                                   // row keys, sort buffer
    t += 2 * align256((size_t)nmax * 4 + 4);                                 // rank sort alt
    t += align256(std::max(radix_temp_bytes(nmax), scan_temp_bytes(nmax + 1)));
    t += 2 * align256((size_t)nV * 4 + 4);                                   // V rank chain
    t += align256(std::max(radix_temp_bytes(nV), scan_temp_bytes(nV + 1)));
    t += 2 * align256((size_t)nmax * 4 + 4) * 2;                             // classify meta/grp
    t += 2 * align256(NCLS * NB * 4) + align256(64 * 8);                     // buckets, bounds
    t += align256((size_t)(nU + 1) * 16) + align256((size_t)(nV + 1) * 16);  // row records
    if (product) g += product_plan(nU, nV, nE).total;
    return {g, t};
}

void layout_graph(DevGraph &g, int64_t nU, int64_t nV, int64_t nE, void *graph_mem,
                  bool product) {
    Carver c{(char *)graph_mem};
    g.nU = nU; g.nV = nV; g.nE = nE;
    int64_t ns[2] = {nU, nV};
    for (int s = 0; s < 2; s++) {
        SideCSR &S = g.side[s];
        int64_t n = ns[s], n1 = n > 0 ? n : 1;
        S.n = n;
        S.off = c.take<int64_t>(n + 1);
        S.adj = c.take<uint32_t>(nE);
        S.md = c.take<uint4>(nE);
        S.id_of_sr = c.take<uint32_t>(n1);
        S.sr_of_id = c.take<uint32_t>(n1);
        S.grank = c.take<uint32_t>(n1);
        S.deg = c.take<uint32_t>(n1);
        S.lo = c.take<uint32_t>(n1);
        S.work = c.take<uint64_t>(n1);
        S.work_nh = c.take<uint64_t>(n1);
        S.pv = c.take<unsigned long long>(n1);
    }
    int64_t n = nU + nV;
    g.warp_list = c.take<AnchorRec>(n + 1);
    g.team_list = c.take<AnchorRec>(n + 1);
    g.ctah_list = c.take<AnchorRec>(n + 1);
    g.dense_jobs = c.take<DenseJob>(n + MAX_SPLIT_JOBS);
    g.groups = c.take<SplitGroup>(MAX_SPLIT_JOBS);
    g.gdone = c.take<uint32_t>(MAX_SPLIT_JOBS);
    g.gpart_cap = (uint32_t)gpart_entries(nE);
    g.gpart = c.take<uint32_t>(g.gpart_cap);
    g.ctr = c.take<uint32_t>(NCTR);
    g.wedges = c.take<unsigned long long>(1);
    g.cls_stats = c.take<unsigned long long>(3 * NCLS);
    g.err = c.take<uint32_t>(1);
    g.scratch = c.take<CountScratch>(1);
    g.prod = product ? product_plan(nU, nV, nE) : ProductPlan{};
    if (g.prod.side >= 0) {
        g.prod_x = (uint16_t *)c.p;
        g.prod_c = (float *)(c.p + g.prod.x_bytes);
        g.prod_cnt = (uint32_t *)(c.p + g.prod.x_bytes + g.prod.c_bytes);
        g.prod_ws = c.p + g.prod.x_bytes + g.prod.c_bytes + g.prod.cnt_bytes;
        c.p += g.prod.total;
    } else {
        g.prod_x = nullptr;
        g.prod_c = nullptr;
        g.prod_cnt = nullptr;
        g.prod_ws = nullptr;
    }
}

namespace {

// The build's temporaries, carved from the caller's block in one fixed
// order (so the two build stages below see the same layout).
struct BuildTemp {
    uint32_t *deg_in[2], *cursorV;
    uint32_t *bufA, *bufB, *bufC, *keys[2];
    uint32_t *ralt_k, *ralt_v, *ralt2_k, *ralt2_v;
    void *ptemp, *ptemp2;
    uint32_t *meta[2], *grp[2];
    ClassifyTemp T;
    int64_t *bounds;
    uint4 *rinfo[2];
};

BuildTemp carve_temp(const DevGraph &g, void *temp_mem) {
    const int64_t nU = g.nU, nV = g.nV, nE = g.nE;
    const int64_t nmax = std::max<int64_t>(std::max(nU, nV), 1);
    Carver c{(char *)temp_mem};
    BuildTemp t;
    t.deg_in[0] = c.take<uint32_t>(nU + 1); t.deg_in[1] = c.take<uint32_t>(nV + 1);
    t.cursorV = c.take<uint32_t>(nV + 1);
    t.bufA = c.take<uint32_t>(nE + 1);   // U-side row keys
    t.bufB = c.take<uint32_t>(nE + 1);   // V-side row keys
    t.bufC = c.take<uint32_t>(nE + 1);   // radix sort alternate buffer (validation: degree replicas)
    t.keys[0] = t.bufA; t.keys[1] = t.bufB;
    t.ralt_k = c.take<uint32_t>(nmax + 1);
    t.ralt_v = c.take<uint32_t>(nmax + 1);
    t.ptemp = c.take<char>(std::max(radix_temp_bytes(nmax), scan_temp_bytes(nmax + 1)));
    t.ralt2_k = c.take<uint32_t>(nV + 1);  // the V side's rank chain, beside the U side's
    t.ralt2_v = c.take<uint32_t>(nV + 1);
    t.ptemp2 = c.take<char>(std::max(radix_temp_bytes(nV), scan_temp_bytes(nV + 1)));
    t.meta[0] = c.take<uint32_t>(nmax + 1); t.meta[1] = c.take<uint32_t>(nmax + 1);
    t.grp[0] = c.take<uint32_t>(nmax + 1); t.grp[1] = c.take<uint32_t>(nmax + 1);
    t.T.bucket_cnt = c.take<uint32_t>(NCLS * NB);
    t.T.bucket_base = c.take<uint32_t>(NCLS * NB);
    t.bounds = c.take<int64_t>(32);
    t.rinfo[0] = c.take<uint4>(nU + 1); t.rinfo[1] = c.take<uint4>(nV + 1);  // per-row records
    return t;
}

// classification of both sides: classes and bucket counts, bucket bases,
// then the class lists and dense jobs
void launch_classes(DevGraph &g, ClassifyTemp T, uint32_t *const *meta, uint32_t *const *grp,
                    cudaStream_t s) {
    const int64_t ns[2] = {g.nU, g.nV};
    for (int sd = 0; sd < 2; sd++) {
        if (ns[sd] == 0) continue;
        T.meta = meta[sd];
        T.grp = grp[sd];
        k_classify<<<grid_for(ns[sd], BT, 4096), BT, 0, s>>>(g.side[sd], sd, T, g); note_launch();
    }
    k_bucket_base<<<1, 32, 0, s>>>(T, g); note_launch();
    cudaMemsetAsync(T.bucket_cnt, 0, NCLS * NB * 4, s);
    for (int sd = 0; sd < 2; sd++) {
        if (ns[sd] == 0) continue;
        T.meta = meta[sd];
        T.grp = grp[sd];
        k_emit<<<grid_for(ns[sd], BT, 2048), BT, 0, s>>>(g.side[sd], sd, T, g); note_launch();
    }
}

}  // namespace

bb_status build_validate(DevGraph &g, const int64_t *rowptr, const int32_t *col, const int8_t *sign,
                         void *temp_mem, cudaStream_t s, const StagedInput *in, uint32_t *verr,
                         uint32_t *pin_err, uint32_t *pin_max) {
    const int64_t nU = g.nU, nV = g.nV, nE = g.nE;
    BuildTemp bt = carve_temp(g, temp_mem);
    uint32_t **deg_in = bt.deg_in, *cursorV = bt.cursorV;
    ClassifyTemp &T = bt.T;
    cudaMemsetAsync(g.err, 0, 4, s);
    cudaMemsetAsync(g.ctr, 0, NCTR * 4, s);
    cudaMemsetAsync(g.wedges, 0, 8, s);
    cudaMemsetAsync(g.cls_stats, 0, 3 * NCLS * 8, s);
    cudaMemsetAsync(cursorV, 0, (size_t)nV * 4, s);
    cudaMemsetAsync(T.bucket_cnt, 0, NCLS * NB * 4, s);
    // V degree replicas in the (not yet used) sort buffer when it has room:
    // up to DEG_COPIES, a power of two
    const int64_t stride = (nV + 64) & ~(int64_t)63;
    uint32_t copies = 1;
    while (copies < DEG_COPIES &&
           (int64_t)(2 * copies) * stride * 4 <= (int64_t)(nE + 1) * 4) copies *= 2;
    uint32_t *degc = copies > 1 ? reinterpret_cast<uint32_t *>(bt.bufC) : deg_in[1];
    cudaMemsetAsync(degc, 0, (size_t)(copies > 1 ? copies * stride : nV) * 4, s);

    // 1. validate + degrees
    if (in) cudaStreamWaitEvent(s, in->rowptr_ready, 0);
    if (nU > 0) k_validate_rows<<<grid_for(nU, BT, 8192), BT, 0, s>>>(rowptr, nU, nE, deg_in[0], g.err, g.ctr + CTR_MAXDEG); note_launch();
    if (nE > 0 && in && in->chunks > 0) {
        for (int c = 0; c < in->chunks; c++) {
            const int64_t lo = in->lo[c], n = in->lo[c + 1] - lo;
            cudaStreamWaitEvent(s, in->ready[c], 0);
            if (n > 0) {
                k_validate_edges<<<grid_for(n, BT, 16384), BT, 0, s>>>(col + lo, sign + lo, n, nV,
                                                                      degc, stride, copies,
                                                                      g.err); note_launch();
            }
        }
    } else if (nE > 0) {
        k_validate_edges<<<grid_for(nE, BT, 16384), BT, 0, s>>>(col, sign, nE, nV, degc, stride,
                                                                copies, g.err); note_launch();
    }
    if (nV > 0) k_max_degree<<<grid_for(nV, BT, 8192), BT, 0, s>>>(degc, stride, copies, deg_in[1], nV,
                                                                   g.ctr + CTR_MAXDEG); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(BB_ERR_CUDA, cudaGetErrorString(e));
    // the one host wait of a build: bounded, creating nothing. With pinned
    // words the two results are copied behind the checks and read after the
    // wait; otherwise they are copied from the idle stream to pageable memory
    uint32_t herr = 0, hmax = 0;
    if (pin_err && pin_max) {
        e = cudaMemcpyAsync(pin_err, g.err, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pin_max, g.ctr + CTR_MAXDEG, 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return report_error(BB_ERR_CUDA, cudaGetErrorString(e));
    }
    bb_status st = wait_stream_bounded(s, "input validation");
    if (st != BB_OK) return st;
    if (pin_err && pin_max) {
        herr = *(volatile uint32_t *)pin_err;
        hmax = *(volatile uint32_t *)pin_max;
    } else {
        e = cudaMemcpyAsync(&herr, g.err, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hmax, g.ctr + CTR_MAXDEG, 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return report_error(BB_ERR_CUDA, cudaGetErrorString(e));
    }
    *verr = herr;
    g.h_maxdeg = hmax;
    g.deg_bits = hmax < (1u << 16) ? 16 : hmax < (1u << 24) ? 24 : 32;
    return BB_OK;
}

void build_rest(DevGraph &g, const int64_t *rowptr, const int32_t *col, const int8_t *sign,
                void *temp_mem, cudaStream_t s, const BuildAux *aux, bool product_only) {
    const int64_t nU = g.nU, nV = g.nV, nE = g.nE;
    BuildTemp bt = carve_temp(g, temp_mem);
    uint32_t **deg_in = bt.deg_in, *cursorV = bt.cursorV;
    uint32_t *bufC = bt.bufC, **keys = bt.keys;
    uint32_t *ralt_k = bt.ralt_k, *ralt_v = bt.ralt_v;
    void *ptemp = bt.ptemp;
    uint32_t **meta = bt.meta, **grp = bt.grp;
    ClassifyTemp &T = bt.T;
    int64_t *bounds = bt.bounds;
    uint4 **rinfo = bt.rinfo;
    // 2. side ranks by (degree, id) and the row offsets in rank order: the
    // U side on s, the V side on the second auxiliary stream when there is
    // one (each with its own sort scratch); then the global priority rank
    int64_t ns[2] = {nU, nV};
    if (aux) {
        cudaEventRecord(aux->fork, s);
        cudaStreamWaitEvent(aux->stream2, aux->fork, 0);
    }
    for (int sd = 0; sd < 2; sd++) {
        int64_t n = ns[sd];
        if (n == 0) {  // an empty side's single offset
            cudaMemsetAsync(g.side[sd].off, 0, 8, s);
            continue;
        }
        SideCSR &S = g.side[sd];
        const cudaStream_t ss = (aux && sd == 1) ? aux->stream2 : s;
        uint32_t *rk = sd ? bt.ralt2_k : ralt_k, *rv = sd ? bt.ralt2_v : ralt_v;
        void *pt = sd ? bt.ptemp2 : ptemp;
        // sort ids by degree (stable => ties by id): reuse id_of_sr / deg as buffers
        k_iota<<<grid_for(n, BT, 8192), BT, 0, ss>>>(S.sr_of_id, n); note_launch();
        cudaMemcpyAsync(S.lo, deg_in[sd], (size_t)n * 4, cudaMemcpyDeviceToDevice, ss);
        radix_sort_pairs_u32(S.lo, S.sr_of_id, rk, rv, n, g.deg_bits, pt, ss);
        cudaMemcpyAsync(rv, S.sr_of_id, (size_t)n * 4, cudaMemcpyDeviceToDevice, ss);
        k_side_rank<<<grid_for(n, BT, 8192), BT, 0, ss>>>(rv, S.lo, n, S); note_launch();
        scan_exclusive_u32_to_i64(S.deg, S.off, n, pt, ss);
    }
    if (aux) {
        cudaEventRecord(aux->join2, aux->stream2);
        cudaStreamWaitEvent(s, aux->join2, 0);
    }
    if (nU > 0) k_global_rank<<<grid_for(nU, BT, 8192), BT, 0, s>>>(g.side[0], g.side[1].deg, nV, 1); note_launch();
    if (nV > 0) k_global_rank<<<grid_for(nV, BT, 8192), BT, 0, s>>>(g.side[1], g.side[0].deg, nU, 0); note_launch();
    g.product_only = product_only;
    if (product_only) return;  // the product path fills its matrices and counts the wedges

    // 3. row fill, row sorts, lo
    if (nU > 0 && nE > 0)
        k_fill<<<grid_for(nE, FILL_EDGES, 4096), FILL_THREADS, 0, s>>>(
            rowptr, col, sign, nU, nE, g.side[0], g.side[1], cursorV, keys[0], keys[1],
            g.err); note_launch();
    // bd[k]: first rank with degree > ROW_LIMS[k]; bd[NLIMS] = n
    for (int sd = 0; sd < 2; sd++)
        if (ns[sd] > 0 && nE > 0) {
            k_row_bounds<<<1, 32, 0, s>>>(g.side[sd].deg, ns[sd], bounds + sd * 16); note_launch();
        }
    // rows above 2048 entries: per-row radix sort (faster there than bitonic);
    // on the auxiliary stream when there is one, beside the other row sorts
    // (the longest rows' sorts would otherwise leave most SMs idle at the end)
    cudaStream_t rs = aux ? aux->stream : s;
    if (aux) {
        cudaEventRecord(aux->fork, s);
        cudaStreamWaitEvent(rs, aux->fork, 0);
        cudaStreamWaitEvent(aux->stream2, aux->fork, 0);
    }
    for (int sd = 0; sd < 2; sd++) {
        if (ns[sd] == 0 || nE == 0) continue;
        const int64_t n_other = ns[1 - sd];
        if (n_other <= (int64_t)BM_MAX_SLICES * BM_RANKS) {
            k_sort_rows_bitmap<<<2 * build_sms(), BM_THREADS, BM_SMEM, rs>>>(
                g.side[sd], keys[sd], bounds + sd * 16, LIM_LONG, NLIMS,
                (uint32_t)n_other, g.err); note_launch();
            continue;
        }
        int key_bits = 1;
        while (key_bits < 32 && ((uint64_t)1 << key_bits) < (uint64_t)(2 * n_other + 2)) key_bits++;
        k_sort_rows_radix<<<1024, RR_THREADS, 0, rs>>>(g.side[sd], keys[sd], bufC,
                                                        bounds + sd * 16, LIM_LONG, NLIMS, key_bits, g.err); note_launch();
    }
    if (aux) cudaEventRecord(aux->join, rs);
    // the shorter rows: U side on s, V side on the second auxiliary stream
    for (int sd = 0; sd < 2; sd++) {
        int64_t n = ns[sd];
        if (n == 0 || nE == 0) continue;
        SideCSR &S = g.side[sd];
        int64_t *bd = bounds + sd * 16;
        const uint32_t *ky = keys[sd];
        const cudaStream_t ss = (aux && sd == 1) ? aux->stream2 : s;
        k_rows_single<<<grid_for(n, BT, 4096), BT, 0, ss>>>(S, ky, bd); note_launch();
        k_sort_rows_sub<2><<<grid_for(n * 2, BT, 8192), BT, 0, ss>>>(S, ky, bd, 0, g.err); note_launch();
        k_sort_rows_sub<4><<<grid_for(n * 4, BT, 8192), BT, 0, ss>>>(S, ky, bd, 1, g.err); note_launch();
        k_sort_rows_sub<8><<<grid_for(n * 8, BT, 8192), BT, 0, ss>>>(S, ky, bd, 2, g.err); note_launch();
        k_sort_rows_sub<16><<<grid_for(n * 16, BT, 8192), BT, 0, ss>>>(S, ky, bd, 3, g.err); note_launch();
        k_sort_rows_sub<32><<<grid_for(n * 32, BT, 8192), BT, 0, ss>>>(S, ky, bd, 4, g.err); note_launch();
        k_sort_rows_warpreg<2><<<2048, 256, 0, ss>>>(S, ky, bd, 5, g.err); note_launch();
        k_sort_rows_warpreg<4><<<2048, 256, 0, ss>>>(S, ky, bd, 6, g.err); note_launch();
        k_sort_rows_warpreg<8><<<2048, 256, 0, ss>>>(S, ky, bd, 7, g.err); note_launch();
        k_sort_rows_warpreg<16><<<2048, 256, 0, ss>>>(S, ky, bd, 8, g.err); note_launch();
        k_sort_rows_smem<2048, 256><<<2048, 256, 2048 * 4, ss>>>(S, ky, bd, 9, g.err); note_launch();
    }
    if (aux) {
        cudaEventRecord(aux->join2, aux->stream2);
        cudaStreamWaitEvent(s, aux->join, 0);
        cudaStreamWaitEvent(s, aux->join2, 0);
    }
    // 3b-4. per-row records, suffix starts and work per anchor. Side sd's
    // descriptor pass reads the other side's records, so each stream
    // computes those of the other side and then its own side's
    // descriptors: U on s, V on the second auxiliary stream when there is
    // one (the two chains are independent).
    if (aux) {
        cudaEventRecord(aux->fork, s);
        cudaStreamWaitEvent(aux->stream2, aux->fork, 0);
    }
    const unsigned md_blocks =
        (unsigned)std::min<int64_t>((nE + edgerows::EDGES - 1) / edgerows::EDGES, 8192);
    for (int sd = 0; sd < 2; sd++) {
        if (ns[sd] == 0) continue;
        const cudaStream_t ss = (aux && sd == 1) ? aux->stream2 : s;
        const int od = 1 - sd;  // the side whose records this side's descriptors read
        if (ns[od] > 0) {
            const int64_t n_other = ns[sd];
            const uint32_t wb = n_other > (int64_t)HUB_WINDOW ? (uint32_t)(n_other - HUB_WINDOW) : 0u;
            k_row_info<<<grid_for(ns[od], BT, 8192), BT, 0, ss>>>(g.side[od], g.side[sd], wb,
                                                                 rinfo[od]); note_launch();
        }
        cudaMemsetAsync(g.side[sd].work, 0, (size_t)ns[sd] * 8, ss);
        cudaMemsetAsync(g.side[sd].work_nh, 0, (size_t)ns[sd] * 8, ss);
        if (nE > 0) {
            k_md_work<<<md_blocks, edgerows::THREADS, 0, ss>>>(g.side[sd], g.side[od], rinfo[od], nE,
                                                              g.wedges, g.err); note_launch();
        }
    }
    if (aux) {
        cudaEventRecord(aux->join2, aux->stream2);
        cudaStreamWaitEvent(s, aux->join2, 0);
    }

    // 5. classes (bucket counts, class counters and statistics were zeroed
    // by the validation)
    launch_classes(g, T, meta, grp, s);
}

size_t classify_temp_bytes(int64_t nU, int64_t nV) {
    const int64_t nmax = std::max<int64_t>(std::max(nU, nV), 1);
    return 4 * align256((size_t)(nmax + 1) * 4) + 2 * align256(NCLS * NB * 4);
}

void classify_graph(DevGraph &g, void *ctemp, cudaStream_t s) {
    const int64_t nmax = std::max<int64_t>(std::max(g.nU, g.nV), 1);
    Carver c{(char *)ctemp};
    uint32_t *meta[2], *grp[2];
    meta[0] = c.take<uint32_t>(nmax + 1); meta[1] = c.take<uint32_t>(nmax + 1);
    grp[0] = c.take<uint32_t>(nmax + 1); grp[1] = c.take<uint32_t>(nmax + 1);
    ClassifyTemp T;
    T.bucket_cnt = c.take<uint32_t>(NCLS * NB);
    T.bucket_base = c.take<uint32_t>(NCLS * NB);
    // class counters, split-group allocators and statistics start afresh;
    // the split-merge counters (gpart, gdone) are zero between counts
    cudaMemsetAsync(g.ctr, 0, CTR_MAXDEG * 4, s);
    cudaMemsetAsync(g.cls_stats, 0, 3 * NCLS * 8, s);
    cudaMemsetAsync(T.bucket_cnt, 0, NCLS * NB * 4, s);
    launch_classes(g, T, meta, grp, s);
}

cudaError_t aux_create(BuildAux &a) {
    cudaError_t e = cudaStreamCreateWithFlags(&a.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a.stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join2, cudaEventDisableTiming);
    return e;
}

void aux_destroy(BuildAux &a) {
    for (cudaStream_t *st : {&a.stream, &a.stream2})
        if (*st) {
            // work still running after the wait limit keeps its stream (leaked)
            if (wait_bounded(*st, "auxiliary stream") == BB_OK) cudaStreamDestroy(*st);
            *st = nullptr;
        }
    for (cudaEvent_t *ev : {&a.fork, &a.join, &a.join2})
        if (*ev) { cudaEventDestroy(*ev); *ev = nullptr; }
}

bb_status build_graph(DevGraph &g, const int64_t *rowptr, const int32_t *col, const int8_t *sign,
                      void *temp_mem, cudaStream_t s, const BuildAux *aux, uint32_t *verr) {
    const bb_status st = build_validate(g, rowptr, col, sign, temp_mem, s, nullptr, verr);
    if (st != BB_OK || *verr) return st;
    build_rest(g, rowptr, col, sign, temp_mem, s, aux);
    return BB_OK;
}

}  // namespace bb
