// prims.cu - device-wide exclusive scan and stable LSD radix sort.
#include "prims.cuh"
#include "common.cuh"

namespace bb {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 4096

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename TIn>
__global__ void k_scan_reduce(const TIn *in, int64_t n, uint64_t *block_sums) {
    __shared__ uint64_t warp_sums[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += (uint64_t)in[i];
    }
    s = warp_sum_u64(s);
    if (lane_id() == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t t = threadIdx.x < SCAN_THREADS / 32 ? warp_sums[threadIdx.x] : 0;
        t = warp_sum_u64(t);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = t;
    }
}

// exclusive scan of one tile (thread-contiguous items) plus a block offset;
// writes out[n] = grand total when it owns the last element
template <typename TIn, typename TOut>
__global__ void k_scan_tile(const TIn *in, TOut *out, int64_t n, const uint64_t *block_offsets) {
    __shared__ uint64_t warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t v[SCAN_ITEMS];
    uint64_t local = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        v[k] = i < n ? (uint64_t)in[i] : 0;
        local += v[k];
    }
    // inclusive warp scan of the per-thread sums (64-bit)
    uint64_t x = local;
    const unsigned lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= (unsigned)d) x += y;
    }
    if (lane == 31) warp_tot[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t t = threadIdx.x < SCAN_THREADS / 32 ? warp_tot[threadIdx.x] : 0;
        uint64_t tx = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(FULL, tx, d);
            if (threadIdx.x >= (unsigned)d) tx += y;
        }
        if (threadIdx.x < SCAN_THREADS / 32) warp_tot[threadIdx.x] = tx - t;  // exclusive
    }
    __syncthreads();
    uint64_t run = block_offsets[blockIdx.x] + warp_tot[threadIdx.x >> 5] + (x - local);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = (TOut)run;
        run += v[k];
        if (i == n - 1) out[n] = (TOut)run;
    }
}

// exclusive scan of n uint64 block sums in place (recursive through temp)
void scan_blocks(uint64_t *sums, int64_t n, uint64_t *temp, cudaStream_t s);

template <typename TIn, typename TOut>
void scan_impl(const TIn *in, TOut *out, int64_t n, void *temp, cudaStream_t s) {
    if (n <= 0) {
        if constexpr (sizeof(TOut) == 8) {
            cudaMemsetAsync(out, 0, sizeof(TOut), s);
        }
        return;
    }
    int64_t nb = ceil_div(n, SCAN_TILE);
    uint64_t *sums = (uint64_t *)temp;
    uint64_t *rest = sums + ceil_div(nb + 1, 32) * 32;
    k_scan_reduce<TIn><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums); note_launch();
    scan_blocks(sums, nb, rest, s);
    k_scan_tile<TIn, TOut><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums); note_launch();
}

void scan_blocks(uint64_t *sums, int64_t n, uint64_t *temp, cudaStream_t s) {
    // exclusive scan in place: scan into sums itself (k_scan_tile reads
    // each element before writing it within the same thread)
    int64_t nb = ceil_div(n, SCAN_TILE);
    uint64_t *bsums = temp;
    uint64_t *rest = bsums + ceil_div(nb + 1, 32) * 32;
    k_scan_reduce<uint64_t><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(sums, n, bsums); note_launch();
    if (nb > 1) {
        scan_blocks(bsums, nb, rest, s);
    } else {
        cudaMemsetAsync(bsums, 0, sizeof(uint64_t), s);
    }
    k_scan_tile<uint64_t, uint64_t><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(sums, sums, n, bsums); note_launch();
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // 4096
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_radix_hist(const uint32_t *keys, int64_t n, int shift, uint64_t *hist,
                             int64_t ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t *keys_in, const uint32_t *vals_in,
                                uint32_t *keys_out, uint32_t *vals_out, int64_t n, int shift,
                                const uint64_t *offsets, int64_t ntiles) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t run[256];
    __shared__ uint64_t base_off[256];
    const int t = threadIdx.x, warp = t >> 5;
    const unsigned lane = lane_id();
    run[t] = 0;
    base_off[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) wcnt[w][t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + (int64_t)r * RS_THREADS + t;
        bool valid = i < n;
        uint32_t k = valid ? keys_in[i] : 0u;
        uint32_t d = valid ? ((k >> shift) & 255u) : 256u + lane;
        unsigned peers = __match_any_sync(FULL, d);
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t sacc = run[t];
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][t];
            wcnt[w][t] = sacc;
            sacc += c;
        }
        run[t] = sacc;
        __syncthreads();
        if (valid) {
            uint64_t pos = base_off[d] + wcnt[warp][d] + rank;
            keys_out[pos] = k;
            vals_out[pos] = vals_in[i];
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) wcnt[w][t] = 0;
        __syncthreads();
    }
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    do {
        m = ceil_div(m, SCAN_TILE);
        total += (size_t)(ceil_div(m + 1, 32) * 32) * sizeof(uint64_t);
    } while (m > 1);
    return total + 1024;
}

void scan_exclusive_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n, void *temp,
                               cudaStream_t s) {
    scan_impl<uint32_t, int64_t>(in, out, n, temp, s);
}

void scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, void *temp,
                        cudaStream_t s) {
    scan_impl<uint64_t, uint64_t>(in, out, n, temp, s);
}

size_t radix_temp_bytes(int64_t n) {
    int64_t ntiles = ceil_div(n > 0 ? n : 1, RS_TILE);
    size_t hist = (size_t)(256 * ntiles + 1) * sizeof(uint64_t);
    return ((hist + 255) & ~(size_t)255) + scan_temp_bytes(256 * ntiles);
}

void radix_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                          int64_t n, int key_bits, void *temp, cudaStream_t s) {
    if (n <= 1) return;
    int64_t ntiles = ceil_div(n, RS_TILE);
    uint64_t *hist = (uint64_t *)temp;
    size_t hist_bytes = (size_t)(256 * ntiles + 1) * sizeof(uint64_t);
    void *scan_tmp = (char *)temp + ((hist_bytes + 255) & ~(size_t)255);
    int passes = (key_bits + 7) / 8;
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_radix_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ki, n, shift, hist, ntiles); note_launch();
        scan_impl<uint64_t, uint64_t>(hist, hist, 256 * ntiles, scan_tmp, s);
        k_radix_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, hist,
                                                                ntiles); note_launch();
        uint32_t *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    if (ki != keys) {
        cudaMemcpyAsync(keys, ki, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    }
}

}  // namespace bb
