// base.cu - BB-Base (Algorithm 1) on the GPU: the paper's baseline, kept to
// measure the gap to the bucket method on the same device.
//
// Algorithm 1 groups, for a pair of same-side vertices, the middle vertices
// of their wedges, and tests every pair of middles explicitly: the
// butterfly on middles v1, v2 is balanced when the two wedges have the same
// sign type (Lemma 1). Here the pairs are the anchor pairs of the bucket
// method (graph.cuh): per anchor w, pass 1 counts the wedges per endpoint u,
// a block scan turns the counts into group offsets, pass 2 writes each
// wedge's type into its endpoint's group (a per-CTA buffer in global
// memory), and pass 3 walks every pair of every group. The work is the
// number of butterflies instead of the number of wedges.
#include <algorithm>
#include <mutex>

#include "graph.cuh"

namespace bb {

namespace {

constexpr int BASE_THREADS = 512;
constexpr uint32_t BASE_DENSE = 16384;  // endpoints per dense window
constexpr uint32_t BASE_HASH = 8192;    // hash slots (u64: endpoint + 1 << 32 | count)

struct BaseSmem {
    union {
        uint32_t cnt[BASE_DENSE];
        unsigned long long tab[BASE_HASH];
    };
    uint32_t off[BASE_DENSE + 1];  // group offsets (exclusive scan), then the end
    uint32_t part[BASE_THREADS / 32];
    uint32_t job;
};

__device__ __forceinline__ int base_hash_slot(unsigned long long *tab, uint32_t shift, uint32_t mask,
                                              uint32_t key, bool insert, uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        unsigned long long cur = *((volatile unsigned long long *)&tab[h]);
        const uint32_t k = (uint32_t)(cur >> 32);
        if (k == key) return (int)h;
        if (k == 0) {
            if (!insert) break;
            const unsigned long long old = atomicCAS(&tab[h], 0ull, (unsigned long long)key << 32);
            if (old == 0ull || (uint32_t)(old >> 32) == key) return (int)h;
        }
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
    return -1;
}

// exclusive scan of n u32 values in place-free form: out[i] = sum of in[< i],
// out[n] = total; one pass of per-thread runs and a warp scan of the parts
template <typename Get>
__device__ __forceinline__ void block_scan_offsets(uint32_t n, uint32_t *out, uint32_t *part,
                                                   Get &&get) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t per = (n + BASE_THREADS - 1) / BASE_THREADS;
    const uint32_t i0 = min(n, (uint32_t)t * per), i1 = min(n, i0 + per);
    uint32_t s = 0;
    for (uint32_t i = i0; i < i1; i++) s += get(i);
    uint32_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) part[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t p = lane < BASE_THREADS / 32 ? part[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, p, d);
            if (lane >= d) p += y;
        }
        if (lane < BASE_THREADS / 32) part[lane] = p;  // inclusive over warps
    }
    __syncthreads();
    uint32_t acc = (warp > 0 ? part[warp - 1] : 0u) + x - s;
    for (uint32_t i = i0; i < i1; i++) {
        out[i] = acc;
        acc += get(i);
    }
    if (t == BASE_THREADS - 1) out[n] = part[BASE_THREADS / 32 - 1];
    __syncthreads();
}

__global__ void __launch_bounds__(BASE_THREADS) k_base(DevGraph G, uint8_t *scratch,
                                                       uint64_t scratch_per_cta,
                                                       unsigned long long *acc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BaseSmem &sm = *reinterpret_cast<BaseSmem *>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = BASE_THREADS / 32;
    uint32_t *err = &G.scratch->err;
    uint8_t *buf = scratch + (uint64_t)blockIdx.x * scratch_per_cta;
    const int64_t nA = G.nU + G.nV;
    unsigned long long bal = 0, tot = 0;
    for (;;) {
        if (t == 0) sm.job = atomicAdd(&G.scratch->job_next[JOB_BASE], 1u);
        __syncthreads();
        const int64_t a = sm.job;
        __syncthreads();
        if (a >= nA) break;
        const int sd = a < G.nU ? 0 : 1;
        const SideCSR &S = sd ? G.side[1] : G.side[0];
        const SideCSR &O = sd ? G.side[0] : G.side[1];
        const uint32_t r = (uint32_t)(sd ? a - G.nU : a);
        const uint64_t W = S.work[r];
        if (W == 0) continue;
        const int64_t rb = S.off[r];
        const uint32_t deg = (uint32_t)(S.off[r + 1] - rb);
        const uint64_t above = (uint64_t)(S.n - r - 1);
        const uint64_t dh = W < above ? W : above;
        const bool dense = above <= BASE_DENSE || dh * 2 >= BASE_HASH;
        uint32_t cap = 32, shift = 27;
        if (!dense)
            while ((uint64_t)cap < 2 * dh + 1) { cap <<= 1; shift--; }
        const uint32_t mask = cap - 1;
        const uint32_t e_lo = r + 1, e_hi = (uint32_t)S.n;
        for (uint32_t e0 = e_lo; e0 < e_hi; e0 += dense ? BASE_DENSE : (e_hi - e_lo)) {
            const uint32_t e1 = dense && e_hi - e0 > BASE_DENSE ? e0 + BASE_DENSE : e_hi;
            const bool clip = dense && (e_hi - e_lo) > BASE_DENSE;
            const uint32_t len = dense ? e1 - e0 : cap;
            if (dense) for (uint32_t i = t; i < len; i += BASE_THREADS) sm.cnt[i] = 0;
            else for (uint32_t i = t; i < cap; i += BASE_THREADS) sm.tab[i] = 0ull;
            __syncthreads();
            auto segment = [&](uint32_t j, int64_t &st, int64_t &en, uint32_t &sw) {
                const uint4 d = S.md[rb + j];
                st = d.x; en = d.z; sw = d.w;
                if (clip) {
                    st = lower_bound_u32(O.adj, st, en, e0 << 1);
                    en = lower_bound_u32(O.adj, st, en, e1 << 1);
                }
            };
            // the group (slot) of an endpoint u
            auto slot_of = [&](uint32_t u, bool insert) -> int {
                if (dense) {
                    const uint32_t idx = u - e0;
                    if (idx >= len) { set_error(err, E_INTERNAL); return -1; }
                    return (int)idx;
                }
                return base_hash_slot(sm.tab, shift, mask, u + 1, insert, err);
            };
            // pass 1: wedges per endpoint
            for (uint32_t j = warp; j < deg; j += nwarps) {
                int64_t st, en; uint32_t sw;
                segment(j, st, en, sw);
                for (int64_t p = st + lane; p < en; p += 32) {
                    const int sl = slot_of(O.adj[p] >> 1, true);
                    if (sl < 0) continue;
                    if (dense) atomicAdd(&sm.cnt[sl], 1u);
                    else atomicAdd(&sm.tab[sl], 1ull);
                }
            }
            __syncthreads();
            // group offsets; the counts become the groups' fill cursors
            if (dense) block_scan_offsets(len, sm.off, sm.part, [&](uint32_t i) { return sm.cnt[i]; });
            else block_scan_offsets(len, sm.off, sm.part, [&](uint32_t i) { return (uint32_t)sm.tab[i]; });
            const uint32_t T = sm.off[len];
            if (T > scratch_per_cta) { set_error(err, E_INTERNAL); break; }
            if (dense) for (uint32_t i = t; i < len; i += BASE_THREADS) sm.cnt[i] = 0;
            else for (uint32_t i = t; i < cap; i += BASE_THREADS) sm.tab[i] &= 0xffffffff00000000ull;
            __syncthreads();
            // pass 2: each wedge's type into its endpoint's group
            for (uint32_t j = warp; j < deg; j += nwarps) {
                int64_t st, en; uint32_t sw;
                segment(j, st, en, sw);
                for (int64_t p = st + lane; p < en; p += 32) {
                    const uint32_t x = O.adj[p];
                    const int sl = slot_of(x >> 1, false);
                    if (sl < 0) continue;
                    const uint32_t k = dense ? atomicAdd(&sm.cnt[sl], 1u)
                                             : (uint32_t)atomicAdd(&sm.tab[sl], 1ull);
                    const uint32_t pos = sm.off[sl] + k;
                    if (pos < T) buf[pos] = (uint8_t)((x ^ sw) & 1u);
                    else set_error(err, E_INTERNAL);
                }
            }
            __syncthreads();
            // pass 3: every pair of middles of every group, tested one by one
            for (uint32_t g = warp; g < len; g += nwarps) {
                const uint32_t g0 = sm.off[g], L = sm.off[g + 1] - g0;
                if (L < 2) continue;
                for (uint32_t i = lane; i + 1 < L; i += 32) {
                    const uint8_t ti = buf[g0 + i];
                    for (uint32_t j = i + 1; j < L; j++) {
                        bal += ti == buf[g0 + j];
                        tot += 1;
                    }
                }
            }
            __syncthreads();
            if (!dense) break;
        }
    }
    bal = warp_sum_u64(bal);
    tot = warp_sum_u64(tot);
    if (lane == 0) {
        if (bal) atomicAdd(&acc[0], bal);
        if (tot) atomicAdd(&acc[1], tot);
    }
}

__global__ void k_max_work(SideCSR S, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < S.n;
         r += (int64_t)gridDim.x * blockDim.x)
        m = S.work[r] > m ? S.work[r] : m;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long y = __shfl_down_sync(FULL, m, d);
        m = y > m ? y : m;
    }
    if (lane_id() == 0 && m) atomicMax(out, m);
}

// grid of k_base, once per device (any thread may count on any device)
constexpr int MAX_DEVICES = 64;
int g_base_blocks[MAX_DEVICES];
std::once_flag g_base_once[MAX_DEVICES];

}  // namespace

int base_blocks() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        dev = 0;
    }
    std::call_once(g_base_once[dev], [dev]() {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, dev);
        cudaFuncSetAttribute(k_base, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BaseSmem));
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_base, BASE_THREADS, sizeof(BaseSmem));
        g_base_blocks[dev] = std::max(1, b) * prop.multiProcessorCount;
    });
    return g_base_blocks[dev];
}

void launch_max_work(const DevGraph &g, unsigned long long *out_dev, cudaStream_t s) {
    cudaMemsetAsync(out_dev, 0, 8, s);
    for (int sd = 0; sd < 2; sd++)
        if (g.side[sd].n > 0) {
            const int64_t blocks = std::min<int64_t>((g.side[sd].n + 255) / 256, 4096);
            k_max_work<<<(unsigned)blocks, 256, 0, s>>>(g.side[sd], out_dev); note_launch();
        }
}

void launch_base(const DevGraph &g, uint8_t *scratch, uint64_t per_cta,
                 unsigned long long *acc_dev, cudaStream_t s) {
    const int blocks = base_blocks();
    cudaMemsetAsync(acc_dev, 0, 16, s);
    cudaMemsetAsync(&g.scratch->job_next[JOB_BASE], 0, 4, s);
    cudaMemsetAsync(&g.scratch->err, 0, 4, s);
    k_base<<<blocks, BASE_THREADS, sizeof(BaseSmem), s>>>(g, scratch, per_cta, acc_dev); note_launch();
}

}  // namespace bb
