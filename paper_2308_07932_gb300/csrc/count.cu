// count.cu - wedge aggregation and the C(.,2) reduction (Algorithm 2's
// counting loop and Lemma 2, made data parallel over anchors as in
// Algorithm 4; the anchor/endpoint roles are described in graph.cuh).
//
// For an anchor w every wedge w - v - u (v a neighbour of w, u in the suffix
// of v's row ranked above both) adds 1 to the symmetric tally of the pair
// (w, u) when sign(w,v) == sign(v,u) (Def. 5) and to the asymmetric tally
// otherwise (Def. 6). Once all of w's wedges are in, each pair with S
// symmetric and A asymmetric wedges adds C(S,2) + C(A,2) balanced and
// C(S+A,2) total butterflies (Lemma 2).
//
// Counter storage per work class:
//   dense  - one u32 per endpoint side rank in shared memory (S in the low
//            16 bits, A in the high 16 bits), for anchors with a small
//            endpoint range; long ranges are walked in windows; very heavy
//            anchors are split over several CTAs whose counters are merged
//            in global memory before the C(.,2) step (C is not additive);
//   hash   - open addressing in shared memory, one u64 per slot
//            (endpoint + 1 in the high half, S | A << 16 in the low half),
//            sized at twice the anchor's distinct-endpoint bound; one table
//            per warp (small anchors) or per CTA.
#include <algorithm>
#include "graph.cuh"

namespace bb {

namespace {

constexpr int DENSE_THREADS = 512;
constexpr int CTAH_THREADS = 512;
constexpr uint32_t CTAH_CAP = 2 * CTA_D_MAX;        // 16384 slots, 128 KiB
constexpr int WARPH_THREADS = 256;                   // 8 warps per CTA
constexpr uint32_t WARPH_CAP = 2 * WARP_D_MAX;      // 1024 slots per warp

__device__ __forceinline__ void acc_add(CountScratch *sc, unsigned long long bal,
                                        unsigned long long tot) {
    if (bal) {
        unsigned long long old = atomicAdd(&sc->acc[0], bal);
        if (old + bal < old) atomicAdd(&sc->acc[1], 1ull);
    }
    if (tot) {
        unsigned long long old = atomicAdd(&sc->acc[2], tot);
        if (old + tot < old) atomicAdd(&sc->acc[3], 1ull);
    }
}

// per-pair contribution of one packed counter (Lemma 2)
__device__ __forceinline__ void pair_terms(uint32_t c, unsigned long long &bal,
                                           unsigned long long &tot) {
    uint32_t S = c & 0xffffu, A = c >> 16;
    bal += c2(S) + c2(A);
    tot += c2(S + A);
}

// block-wide sum of two u64 values, result valid in thread 0
template <int THREADS>
__device__ __forceinline__ void block_sum2(unsigned long long &a, unsigned long long &b) {
    __shared__ unsigned long long ra[THREADS / 32], rb[THREADS / 32];
    a = warp_sum_u64(a);
    b = warp_sum_u64(b);
    if (lane_id() == 0) { ra[threadIdx.x >> 5] = a; rb[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < THREADS / 32 ? ra[threadIdx.x] : 0ull;
        b = threadIdx.x < THREADS / 32 ? rb[threadIdx.x] : 0ull;
        a = warp_sum_u64(a);
        b = warp_sum_u64(b);
    }
    __syncthreads();
}

// Walk the wedges of the anchor whose row starts at rb in side S, over its
// middles [m0, m1), batches of 32 middles taken by this warp starting at
// batch `first` with stride `stride`. With CLIP, only endpoints whose side
// rank lies in [e0, e1) are visited. add(u_side_rank, asymmetric) per wedge.
//
// Each batch is flattened: lane j holds middle j's suffix (start, length),
// a warp scan gives every wedge of the batch an index, and each lane finds
// the middle of its wedge by binary search over the 32 running sums.
template <bool CLIP, typename F>
__device__ __forceinline__ void walk(const SideCSR &S, const SideCSR &O, int64_t rb, uint32_t m0,
                                     uint32_t m1, uint32_t e0, uint32_t e1, uint32_t first,
                                     uint32_t stride, F &&add) {
    const unsigned lane = lane_id();
    for (uint32_t mb = m0 + first * 32u; mb < m1; mb += stride * 32u) {
        uint32_t j = mb + lane;
        uint32_t len = 0, sw = 0;
        long long st = 0;
        if (j < m1) {
            uint32_t ent = S.adj[rb + j];
            uint32_t v = ent >> 1;
            sw = ent & 1u;
            long long ve = O.off[v + 1];
            st = O.off[v] + S.sfx[rb + j];
            if (CLIP) {
                long long a = lower_bound_u32(O.adj, st, ve, e0 << 1);
                ve = lower_bound_u32(O.adj, a, ve, e1 << 1);
                st = a;
            }
            len = (uint32_t)(ve - st);
        }
        uint32_t incl = warp_incl_scan(len);
        uint32_t total = __shfl_sync(FULL, incl, 31);
        uint32_t excl = incl - len;
        for (uint32_t k = 0; k < total; k += 32) {
            uint32_t i = k + lane;
            uint32_t m = 0;
#pragma unroll
            for (int b = 16; b >= 1; b >>= 1) {
                uint32_t c = __shfl_sync(FULL, incl, m + b - 1);
                if (c <= i) m += b;
            }
            long long stm = __shfl_sync(FULL, st, m);
            uint32_t exm = __shfl_sync(FULL, excl, m);
            uint32_t swm = __shfl_sync(FULL, sw, m);
            if (i < total) {
                uint32_t x = O.adj[stm + (i - exm)];
                add(x >> 1, (x ^ swm) & 1u);
            }
        }
    }
}

// insert-or-increment in a shared-memory table of 2^(32-shift) u64 slots
__device__ __forceinline__ void hash_add(unsigned long long *tab, uint32_t shift, uint32_t mask,
                                         uint32_t key, uint32_t inc, uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        unsigned long long cur = *((volatile unsigned long long *)&tab[h]);
        uint32_t k = (uint32_t)(cur >> 32);
        if (k == key) { atomicAdd(&tab[h], (unsigned long long)inc); return; }
        if (k == 0) {
            unsigned long long want = ((unsigned long long)key << 32) | inc;
            unsigned long long old = atomicCAS(&tab[h], 0ull, want);
            if (old == 0ull) return;
            if ((uint32_t)(old >> 32) == key) { atomicAdd(&tab[h], (unsigned long long)inc); return; }
        }
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
}

__device__ __forceinline__ void table_geometry(uint64_t dh, uint32_t min_cap, uint32_t &cap,
                                               uint32_t &shift) {
    cap = min_cap;
    shift = 32 - (31 - __clz(min_cap));
    while ((uint64_t)cap < 2 * dh) { cap <<= 1; shift--; }
}

// ------------------------------------------------------------ dense class
__global__ void __launch_bounds__(DENSE_THREADS) k_dense(DevGraph G) {
    extern __shared__ uint32_t cnt[];
    __shared__ uint32_t s_job, s_last;
    const uint32_t njobs = G.ctr[CTR_DENSE];
    const uint32_t warp = threadIdx.x >> 5, nwarps = DENSE_THREADS / 32;
    CountScratch *sc = G.scratch;
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(&sc->job_next[CLS_DENSE], 1u);
        __syncthreads();
        const uint32_t jid = s_job;
        if (jid >= njobs) break;
        const DenseJob J = G.dense_jobs[jid];
        const int sd = J.anchor & 1u;
        const uint32_t r = J.anchor >> 1;
        const SideCSR S = sd ? G.side[1] : G.side[0];
        const SideCSR O = sd ? G.side[0] : G.side[1];
        const int64_t rb = S.off[r];
        const uint32_t e_lo = r + 1, e_hi = (uint32_t)S.n;
        const bool windows = (e_hi - e_lo) > DENSE_CAP;
        for (uint32_t e0 = e_lo; e0 < e_hi; e0 += DENSE_CAP) {
            const uint32_t e1 = e_hi - e0 > DENSE_CAP ? e0 + DENSE_CAP : e_hi;
            const uint32_t len = e1 - e0;
            for (uint32_t i = threadIdx.x; i < len; i += DENSE_THREADS) cnt[i] = 0;
            __syncthreads();
            auto add = [&](uint32_t u, uint32_t asym) {
                uint32_t idx = u - e0;
                if (idx < len) atomicAdd(&cnt[idx], asym ? INC_ASYM : INC_SYM);
                else set_error(&sc->err, E_INTERNAL);
            };
            if (windows) walk<true>(S, O, rb, J.m0, J.m1, e0, e1, warp, nwarps, add);
            else walk<false>(S, O, rb, J.m0, J.m1, e0, e1, warp, nwarps, add);
            __syncthreads();
            unsigned long long bal = 0, tot = 0;
            if (J.group == NO_GROUP) {
                for (uint32_t i = threadIdx.x; i < len; i += DENSE_THREADS) pair_terms(cnt[i], bal, tot);
            } else {
                const SplitGroup grp = G.groups[J.group];
                uint32_t *part = G.gpart + grp.goff;
                for (uint32_t i = threadIdx.x; i < len; i += DENSE_THREADS)
                    if (cnt[i]) atomicAdd(&part[i], cnt[i]);
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t ticket = atomicAdd(&G.gdone[J.group], 1u);
                    s_last = ticket == grp.parts - 1 ? 1u : 0u;
                }
                __syncthreads();
                if (s_last) {
                    __threadfence();
                    for (uint32_t i = threadIdx.x; i < len; i += DENSE_THREADS) {
                        uint32_t c = __ldcg(&part[i]);
                        pair_terms(c, bal, tot);
                        part[i] = 0;
                    }
                    if (threadIdx.x == 0) G.gdone[J.group] = 0;
                }
            }
            block_sum2<DENSE_THREADS>(bal, tot);
            if (threadIdx.x == 0) acc_add(sc, bal, tot);
        }
    }
}

// --------------------------------------------------------- CTA hash class
__global__ void __launch_bounds__(CTAH_THREADS) k_ctah(DevGraph G) {
    extern __shared__ unsigned long long tab[];
    __shared__ uint32_t s_job;
    const uint32_t njobs = G.ctr[CTR_CTAH];
    const uint32_t warp = threadIdx.x >> 5, nwarps = CTAH_THREADS / 32;
    CountScratch *sc = G.scratch;
    for (uint32_t i = threadIdx.x; i < CTAH_CAP; i += CTAH_THREADS) tab[i] = 0ull;
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(&sc->job_next[CLS_CTAH], 1u);
        __syncthreads();
        const uint32_t jid = s_job;
        if (jid >= njobs) break;
        const uint32_t anchor = G.ctah_list[jid];
        const int sd = anchor & 1u;
        const uint32_t r = anchor >> 1;
        const SideCSR S = sd ? G.side[1] : G.side[0];
        const SideCSR O = sd ? G.side[0] : G.side[1];
        const int64_t rb = S.off[r];
        const uint32_t deg = (uint32_t)(S.off[r + 1] - rb);
        uint64_t W = S.work[r], above = (uint64_t)(S.n - r - 1);
        uint32_t cap, shift;
        table_geometry(W < above ? W : above, 64, cap, shift);
        if (cap > CTAH_CAP) { cap = CTAH_CAP; shift = 32 - 14; }
        const uint32_t mask = cap - 1;
        uint32_t *err = &sc->err;
        walk<false>(S, O, rb, 0, deg, 0, 0, warp, nwarps, [&](uint32_t u, uint32_t asym) {
            hash_add(tab, shift, mask, u + 1, asym ? INC_ASYM : INC_SYM, err);
        });
        __syncthreads();
        unsigned long long bal = 0, tot = 0;
        for (uint32_t i = threadIdx.x; i < cap; i += CTAH_THREADS) {
            unsigned long long t = tab[i];
            if (t) { pair_terms((uint32_t)t, bal, tot); tab[i] = 0ull; }
        }
        block_sum2<CTAH_THREADS>(bal, tot);
        if (threadIdx.x == 0) acc_add(sc, bal, tot);
    }
}

// -------------------------------------------------------- warp hash class
__global__ void __launch_bounds__(WARPH_THREADS) k_warph(DevGraph G) {
    extern __shared__ unsigned long long tabs[];
    const uint32_t warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    unsigned long long *tab = tabs + (size_t)warp * WARPH_CAP;
    for (uint32_t i = lane; i < WARPH_CAP; i += 32) tab[i] = 0ull;
    __syncwarp();
    const uint32_t n = G.ctr[CTR_WARP];
    const uint32_t gw = (blockIdx.x * WARPH_THREADS + threadIdx.x) >> 5;
    const uint32_t GW = (gridDim.x * WARPH_THREADS) >> 5;
    CountScratch *sc = G.scratch;
    uint32_t *err = &sc->err;
    unsigned long long bal = 0, tot = 0;
    for (uint32_t idx = gw; idx < n; idx += GW) {
        const uint32_t anchor = G.warp_list[idx];
        const int sd = anchor & 1u;
        const uint32_t r = anchor >> 1;
        const SideCSR S = sd ? G.side[1] : G.side[0];
        const SideCSR O = sd ? G.side[0] : G.side[1];
        const int64_t rb = S.off[r];
        const uint32_t deg = (uint32_t)(S.off[r + 1] - rb);
        uint64_t W = S.work[r], above = (uint64_t)(S.n - r - 1);
        uint32_t cap, shift;
        table_geometry(W < above ? W : above, 32, cap, shift);
        if (cap > WARPH_CAP) { cap = WARPH_CAP; shift = 32 - 10; }
        const uint32_t mask = cap - 1;
        walk<false>(S, O, rb, 0, deg, 0, 0, 0, 1, [&](uint32_t u, uint32_t asym) {
            hash_add(tab, shift, mask, u + 1, asym ? INC_ASYM : INC_SYM, err);
        });
        __syncwarp();
        for (uint32_t i = lane; i < cap; i += 32) {
            unsigned long long t = tab[i];
            if (t) { pair_terms((uint32_t)t, bal, tot); tab[i] = 0ull; }
        }
        __syncwarp();
    }
    block_sum2<WARPH_THREADS>(bal, tot);
    if (threadIdx.x == 0) acc_add(sc, bal, tot);
}

// ------------------------------------------------------------ sign flips
__global__ void k_flip(DevGraph G, const int64_t *edge_idx, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = edge_idx[t];
        if (e < 0 || e >= G.nE) { set_error(&G.scratch->err, E_INTERNAL); continue; }
        int64_t lo = 0, hi = G.nU;  // u = last row with rowptr[u] <= e
        while (hi - lo > 1) {
            int64_t m = (lo + hi) >> 1;
            if (G.rowptr[m] <= e) lo = m; else hi = m;
        }
        uint32_t ru = G.side[0].sr_of_id[lo];
        uint32_t rv = G.side[1].sr_of_id[G.col[e]];
        const SideCSR &U = G.side[0];
        const SideCSR &V = G.side[1];
        int64_t p = lower_bound_u32(U.adj, U.off[ru], U.off[ru + 1], rv << 1);
        int64_t q = lower_bound_u32(V.adj, V.off[rv], V.off[rv + 1], ru << 1);
        atomicXor(&U.adj[p], 1u);
        atomicXor(&V.adj[q], 1u);
    }
}

struct LaunchCfg {
    int dense_blocks = 0, ctah_blocks = 0, warph_blocks = 0;
};

LaunchCfg g_cfg;
int g_cfg_device = -1;

void init_cfg() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_cfg_device == dev) return;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    const int sms = prop.multiProcessorCount;
    size_t dense_smem = DENSE_CAP * 4, ctah_smem = CTAH_CAP * 8,
           warph_smem = (size_t)(WARPH_THREADS / 32) * WARPH_CAP * 8;
    cudaFuncSetAttribute(k_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem);
    cudaFuncSetAttribute(k_ctah, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctah_smem);
    cudaFuncSetAttribute(k_warph, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)warph_smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dense, DENSE_THREADS, dense_smem);
    g_cfg.dense_blocks = std::max(1, b) * sms;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ctah, CTAH_THREADS, ctah_smem);
    g_cfg.ctah_blocks = std::max(1, b) * sms;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_warph, WARPH_THREADS, warph_smem);
    g_cfg.warph_blocks = std::max(1, b) * sms;
    g_cfg_device = dev;
}

}  // namespace

void count_init() { init_cfg(); build_init(); }

void launch_count(const DevGraph &g, cudaStream_t s, int64_t *per_vertex_dev) {
    (void)per_vertex_dev;
    init_cfg();
    cudaMemsetAsync(g.scratch, 0, sizeof(CountScratch), s);
    k_dense<<<g_cfg.dense_blocks, DENSE_THREADS, DENSE_CAP * 4, s>>>(g);
    k_ctah<<<g_cfg.ctah_blocks, CTAH_THREADS, CTAH_CAP * 8, s>>>(g);
    k_warph<<<g_cfg.warph_blocks, WARPH_THREADS, (WARPH_THREADS / 32) * WARPH_CAP * 8, s>>>(g);
}

void launch_flip(DevGraph &g, const int64_t *edge_idx_dev, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_flip<<<(unsigned)blocks, 256, 0, s>>>(g, edge_idx_dev, n);
}

}  // namespace bb
