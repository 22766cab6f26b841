// pervertex.cu - balanced butterflies containing each vertex (the quantity
// Algorithm 3 computes for one vertex), for every vertex at once, and
// containing each edge.
//
// Each balanced butterfly is tallied at exactly one pair (w, u) of same-side
// vertices (w the anchor, u the higher-priority one; see graph.cuh) and has
// two middles of the same wedge type. A pair with S symmetric and A
// asymmetric middles holds C(S,2) + C(A,2) balanced butterflies: every one
// contains w and u, and a middle of type t lies in cnt_t - 1 of them (it
// pairs with each other middle of its type). Per anchor the kernel tallies
// the pairs (pass 1), walks the wedges again reading the final tallies and
// adds cnt_t - 1 to each middle (pass 2), then adds each pair's balanced
// count to u and their sum to w.
//
// The same two passes give per-edge counts (the paper's edge-level
// extension): a middle v of type t at pair (w, u) puts its cnt_t - 1
// balanced butterflies on the edges w-v and v-u as well, accumulated per
// adjacency entry of each side and summed per input edge at the end.
//
// This runs only when per-vertex or per-edge counts are requested, after
// the regular count. Warp-class anchors are walked one per warp (k_pv_warp),
// the others one per CTA, one warp per middle (k_pv): with a single
// 512-thread CTA per SM the coalesced reads of a warp per middle beat a
// lane walker here.
#include <algorithm>
#include <mutex>
#include "graph.cuh"

namespace bb {

namespace {

// Two instances of k_pv: dense-class and CTA-hash anchors in 512-thread
// CTAs over 96 KiB of counters (two CTAs per SM; the hybrid hash then holds
// 8,192 slots, enough for every CTA-hash anchor), and team-class anchors,
// whose below-window endpoints fit a TEAM_CAP-slot hash by construction, in
// 128-thread CTAs over 16 KiB (several CTAs per SM).
constexpr int PV_THREADS = 512;
constexpr uint32_t PV_DENSE_CAP = 24576;  // dense counters (96 KiB)
constexpr int PVT_THREADS = 128;
constexpr uint32_t PVT_WORDS = HUB_WINDOW + 2 * TEAM_CAP;  // hub window + TEAM_CAP hash slots

constexpr uint32_t pow2_floor(uint32_t x) {
    uint32_t p = 1;
    while (p <= x / 2) p <<= 1;
    return p;
}

// every CTA-hash anchor (below-window endpoints < CTAH_CAP / 2) fits the
// heavy instance's hybrid hash at load <= 0.8
static_assert(pow2_floor((PV_DENSE_CAP - HUB_WINDOW) / 2) >= CTAH_CAP / 2 * 5 / 4 + 1,
              "CTA-hash anchors would fall back to dense windows");

template <int TH, uint32_t WORDS>
struct PvSmem {
    uint32_t cnt[WORDS];  // dense counters, or the hub window then the hash
    unsigned long long red[TH / 32];
    uint32_t job;
};

__device__ __forceinline__ uint32_t pv_hash_add(unsigned long long *tab, uint32_t shift,
                                                uint32_t mask, uint32_t key, uint32_t inc,
                                                uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        unsigned long long cur = *((volatile unsigned long long *)&tab[h]);
        uint32_t k = (uint32_t)(cur >> 32);
        if (k == key) { atomicAdd(&tab[h], (unsigned long long)inc); return 0; }
        if (k == 0) {
            unsigned long long old = atomicCAS(&tab[h], 0ull, ((unsigned long long)key << 32) | inc);
            if (old == 0ull) return 0;
            if ((uint32_t)(old >> 32) == key) { atomicAdd(&tab[h], (unsigned long long)inc); return 0; }
        }
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
    return 0;
}

__device__ __forceinline__ uint32_t pv_hash_find(const unsigned long long *tab, uint32_t shift,
                                                 uint32_t mask, uint32_t key, uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const unsigned long long cur = tab[h];
        if ((uint32_t)(cur >> 32) == key) return (uint32_t)cur;
        if (cur == 0ull) break;
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
    return 0;
}

// What k_pv accumulates: per-vertex counts (into each side's pv array)
// and/or per-edge counts (into pe[side][position of the entry in that
// side's adjacency]; null when not wanted).
struct PvOut {
    int vertex;
    unsigned long long *pe[2];
};

template <int TH, uint32_t WORDS, bool TEAM>
__global__ void __launch_bounds__(TH) k_pv(DevGraph G, PvOut out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PvSmem<TH, WORDS> &sm = *reinterpret_cast<PvSmem<TH, WORDS> *>(smem_raw);
    // hash slots after the window: the largest power of two that fits
    constexpr uint32_t HYB_CAP = pow2_floor((WORDS - HUB_WINDOW) / 2);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = TH / 32;
    uint32_t *err = &G.scratch->err;
    // team anchors, or the dense and CTA-hash classes (warp-class anchors go
    // to k_pv_warp); a split dense anchor is taken once, at its first part
    const uint32_t nT = G.ctr[CTR_TEAM], nC = G.ctr[CTR_CTAH], nD = G.ctr[CTR_DENSE];
    const uint32_t nJ = TEAM ? nT : nD + nC;
    for (;;) {
        if (t == 0) sm.job = atomicAdd(&G.scratch->job_next[TEAM ? JOB_PV_TEAM : JOB_PER_VERTEX], 1u);
        __syncthreads();
        const uint32_t jb = sm.job;
        __syncthreads();
        if (jb >= nJ) break;
        // heaviest first: dense jobs, then CTA-hash anchors
        uint32_t packed;
        if (TEAM) {
            packed = G.team_list[jb].anchor;
        } else if (jb < nD) {
            const DenseJob &J = G.dense_jobs[jb];
            if (J.m0 != 0) continue;
            packed = J.anchor;
        } else {
            packed = G.ctah_list[jb - nD].anchor;
        }
        const int sd = (int)(packed & 1u);
        const SideCSR &S = sd ? G.side[1] : G.side[0];
        const SideCSR &O = sd ? G.side[0] : G.side[1];
        unsigned long long *peS = out.pe[sd], *peO = out.pe[1 - sd];
        const uint32_t r = packed >> 1;
        const uint64_t W = S.work[r];
        if (W == 0) continue;
        const int64_t rb = S.off[r];
        const uint32_t deg = (uint32_t)(S.off[r + 1] - rb);
        const uint32_t ns = (uint32_t)S.n;
        // hybrid layout: the endpoints in the hub window (the top HUB_WINDOW
        // ranks, those above the anchor) in dense counters, the ones below
        // it in a hash sized by their count; dense layout (when that hash
        // would not fit): counters over the whole endpoint range, walked in
        // windows of the counter capacity when it is longer
        const uint32_t wb = ns > HUB_WINDOW ? ns - HUB_WINDOW : 0u;
        const uint32_t wlo = wb > r + 1 ? wb : r + 1;  // first endpoint in the window
        const uint32_t wlen = ns - wlo;
        const uint64_t above_nh = (uint64_t)(wlo - (r + 1));
        const uint64_t wnh = S.work_nh[r];
        const uint64_t need = (wnh < above_nh ? wnh : above_nh) * 5 / 4 + 1;
        // an anchor of degree above MAX_DEGREE (wide) needs 32-bit S and A:
        // dense windows of half the length, S in the first half of the
        // counters and A in the second (pass 2 reads only final tallies, so
        // two separate arrays suffice)
        const bool wide = deg > MAX_DEGREE;
        const bool hybrid = !wide && need <= HYB_CAP;
        constexpr uint32_t HALF = WORDS / 2;
        const uint32_t span = wide ? HALF : WORDS;
        if (TEAM && !hybrid) {  // impossible for a team-class anchor
            set_error(err, E_INTERNAL);
            continue;
        }
        uint32_t cap = 32, shift = 27;
        if (hybrid)
            while ((uint64_t)cap < need) { cap <<= 1; shift--; }
        const uint32_t mask = cap - 1;
        unsigned long long *tab = reinterpret_cast<unsigned long long *>(sm.cnt + HUB_WINDOW);
        unsigned long long wsum = 0;  // balanced butterflies containing the anchor
        const uint32_t e_lo = r + 1, e_hi = ns;
        for (uint32_t e0 = e_lo; e0 < e_hi; e0 += hybrid ? (e_hi - e_lo) : span) {
            const uint32_t e1 = !hybrid && e_hi - e0 > span ? e0 + span : e_hi;
            const bool clip = !hybrid && (e_hi - e_lo) > span;
            const uint32_t len = hybrid ? wlen : e1 - e0;
            for (uint32_t i = t; i < len; i += TH) sm.cnt[i] = 0;
            if (wide)
                for (uint32_t i = t; i < len; i += TH) sm.cnt[HALF + i] = 0;
            if (hybrid)
                for (uint32_t i = t; i < cap; i += TH) tab[i] = 0ull;
            __syncthreads();
            // segment of middle j's row: the wedge suffix, clipped to [e0, e1)
            auto segment = [&](uint32_t j, int64_t &st, int64_t &en, uint32_t &sw, uint32_t &v) {
                const uint4 d = S.md[rb + j];
                st = d.x; en = d.z; sw = d.w;
                v = S.adj[rb + j] >> 1;
                if (clip) {
                    st = lower_bound_u32(O.adj, st, en, e0 << 1);
                    en = lower_bound_u32(O.adj, st, en, e1 << 1);
                }
            };
            // counter index of endpoint u (>= len: in the hash)
            auto index = [&](uint32_t u) -> uint32_t {
                if (hybrid) return u >= wlo ? u - wlo : 0xffffffffu;
                const uint32_t idx = u - e0;
                if (idx >= len) set_error(err, E_INTERNAL);
                return idx;
            };
            // pass 1: tally (one warp per middle, coalesced reads of its suffix)
            for (uint32_t j = warp; j < deg; j += nwarps) {
                int64_t st, en; uint32_t sw, v;
                segment(j, st, en, sw, v);
                for (int64_t p = st + lane; p < en; p += 32) {
                    const uint32_t x = O.adj[p];
                    const uint32_t u = x >> 1;
                    const uint32_t asym = (x ^ sw) & 1u;
                    const uint32_t inc = asym ? INC_ASYM : INC_SYM;
                    const uint32_t idx = index(u);
                    if (wide) { if (idx < len) atomicAdd(&sm.cnt[asym * HALF + idx], 1u); }
                    else if (idx < len) atomicAdd(&sm.cnt[idx], inc);
                    else if (hybrid) pv_hash_add(tab, shift, mask, u + 1, inc, err);
                }
            }
            __syncthreads();
            // pass 2: each middle v of type t lies in cnt_t - 1 balanced
            // butterflies of its pair (w, u), and so do the edges w-v and v-u
            for (uint32_t j = warp; j < deg; j += nwarps) {
                int64_t st, en; uint32_t sw, v;
                segment(j, st, en, sw, v);
                unsigned long long msum = 0;
                for (int64_t p = st + lane; p < en; p += 32) {
                    const uint32_t x = O.adj[p];
                    const uint32_t u = x >> 1;
                    const uint32_t idx = index(u);
                    uint32_t c = 0, ct;
                    if (wide) {
                        ct = idx < len ? sm.cnt[((x ^ sw) & 1u) * HALF + idx] : 0u;
                    } else {
                        if (idx < len) c = sm.cnt[idx];
                        else if (hybrid) c = pv_hash_find(tab, shift, mask, u + 1, err);
                        ct = ((x ^ sw) & 1u) ? (c >> 16) : (c & 0xffffu);
                    }
                    const unsigned long long k = ct > 0 ? ct - 1 : 0;
                    msum += k;
                    if (peO && k) atomicAdd(&peO[p], k);   // edge v-u
                }
                msum = warp_sum_u64(msum);
                if (lane == 0 && msum) {
                    if (out.vertex) atomicAdd(&O.pv[v], msum);
                    if (peS) atomicAdd(&peS[rb + j], msum);  // edge w-v
                }
            }
            __syncthreads();
            if (!out.vertex) continue;
            // each pair's balanced butterflies contain both of its endpoints
            const uint32_t ubase = hybrid ? wlo : e0;
            for (uint32_t i = t; i < len; i += TH) {
                const uint32_t c = sm.cnt[i];
                const unsigned long long b =
                    wide ? c2(c) + c2(sm.cnt[HALF + i]) : c2(c & 0xffffu) + c2(c >> 16);
                if (b) { atomicAdd(&S.pv[ubase + i], b); wsum += b; }
            }
            if (hybrid)
                for (uint32_t i = t; i < cap; i += TH) {
                    const unsigned long long x = tab[i];
                    if (!x) continue;
                    const uint32_t c = (uint32_t)x;
                    const unsigned long long b = c2(c & 0xffffu) + c2(c >> 16);
                    if (b) { atomicAdd(&S.pv[(uint32_t)(x >> 32) - 1u], b); wsum += b; }
                }
            __syncthreads();
        }
        if (out.vertex) {
            wsum = warp_sum_u64(wsum);
            if (lane == 0) sm.red[warp] = wsum;
            __syncthreads();
            if (t == 0) {
                unsigned long long tot = 0;
                for (int k = 0; k < nwarps; k++) tot += sm.red[k];
                if (tot) atomicAdd(&S.pv[r], tot);
            }
        }
        __syncthreads();
    }
}

// Warp-class anchors (degree <= 255, at most WARP_W_MAX wedges), one per
// warp, with the count's counter layout: the hub window in 16-bit fields
// (S in bits 0..7, A in bits 8..15) and a 256-slot hash for the endpoints
// below it (every endpoint when the anchor has at most WARP_SMALL_W
// wedges). Pass 1 tallies, pass 2 walks each middle's suffix reading the
// final tallies, then the pairs' C(S,2) + C(A,2) go to both endpoints.
constexpr int PVW_THREADS = 256;
constexpr uint32_t PVW_CAP = 256;

struct alignas(16) PvWarpSmem {
    uint32_t win[HUB_WINDOW / 2];
    unsigned long long tab[PVW_CAP];
};

__global__ void __launch_bounds__(PVW_THREADS) k_pv_warp(DevGraph G, PvOut out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PvWarpSmem &sm = reinterpret_cast<PvWarpSmem *>(smem_raw)[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    uint32_t *err = &G.scratch->err;
    for (uint32_t i = lane; i < HUB_WINDOW / 2; i += 32) sm.win[i] = 0;
    for (uint32_t i = lane; i < PVW_CAP; i += 32) sm.tab[i] = 0ull;
    __syncwarp();
    const uint32_t n = G.ctr[CTR_WARP];
    const uint32_t gw = (blockIdx.x * PVW_THREADS + threadIdx.x) >> 5;
    const uint32_t GW = (gridDim.x * PVW_THREADS) >> 5;
    for (uint32_t idx = gw; idx < n; idx += GW) {
        const AnchorRec rec = G.warp_list[idx];
        const int sd = (int)(rec.anchor & 1u);
        const SideCSR &S = sd ? G.side[1] : G.side[0];
        const SideCSR &O = sd ? G.side[0] : G.side[1];
        unsigned long long *peS = out.pe[sd], *peO = out.pe[1 - sd];
        const uint32_t r = rec.anchor >> 1, deg = rec.deg;
        const int64_t rb = rec.rb;
        const uint64_t W = rec.W;
        const uint64_t above = (uint64_t)(S.n - r - 1);
        const bool all_hash = W <= WARP_SMALL_W;
        const uint32_t wb = S.n > (int64_t)HUB_WINDOW ? (uint32_t)(S.n - HUB_WINDOW) : 0u;
        const uint64_t above_nh = wb > r + 1 ? (uint64_t)wb - r - 1 : 0;
        uint64_t need = all_hash ? (W < above ? W : above) : (rec.wnh < above_nh ? rec.wnh : above_nh);
        uint32_t cap = 32, shift = 27;
        while ((uint64_t)cap < 2 * need + 1 && cap < PVW_CAP) { cap <<= 1; shift--; }
        const uint32_t mask = cap - 1;
        uint32_t wmin = HUB_WINDOW;
        // endpoint u (side rank) -> its window index, or HUB_WINDOW if hashed
        auto win_index = [&](uint32_t u) -> uint32_t {
            if (all_hash || u < wb) return HUB_WINDOW;
            const uint32_t wi = u - wb;
            if (wi >= HUB_WINDOW) { set_error(err, E_INTERNAL); return HUB_WINDOW; }
            return wi;
        };
        // pass 1: tallies
        for (uint32_t j = 0; j < deg; j++) {
            const uint4 d = S.md[rb + j];
            for (uint32_t p = d.x + lane; p < d.z; p += 32) {
                const uint32_t x = O.adj[p];
                const uint32_t u = x >> 1, asym = (x ^ d.w) & 1u;
                const uint32_t wi = win_index(u);
                if (wi < HUB_WINDOW) {
                    wmin = wi < wmin ? wi : wmin;
                    atomicAdd(&sm.win[wi >> 1], (1u + asym * 255u) << ((wi & 1u) << 4));
                } else {
                    pv_hash_add(sm.tab, shift, mask, u + 1, asym ? INC_ASYM : INC_SYM, err);
                }
            }
        }
        __syncwarp();
        // pass 2: a middle of type t lies in cnt_t - 1 balanced butterflies of
        // each of its pairs, and so do the edges w-v and v-u
        for (uint32_t j = 0; j < deg; j++) {
            const uint4 d = S.md[rb + j];
            unsigned long long msum = 0;
            for (uint32_t p = d.x + lane; p < d.z; p += 32) {
                const uint32_t x = O.adj[p];
                const uint32_t u = x >> 1, asym = (x ^ d.w) & 1u;
                const uint32_t wi = win_index(u);
                uint32_t ct;
                if (wi < HUB_WINDOW) {
                    const uint32_t c = (sm.win[wi >> 1] >> ((wi & 1u) << 4)) & 0xffffu;
                    ct = asym ? (c >> 8) : (c & 0xffu);
                } else {
                    const uint32_t c = pv_hash_find(sm.tab, shift, mask, u + 1, err);
                    ct = asym ? (c >> 16) : (c & 0xffffu);
                }
                const unsigned long long k = ct > 0 ? ct - 1 : 0;
                msum += k;
                if (peO && k) atomicAdd(&peO[p], k);  // edge v-u
            }
            msum = warp_sum_u64(msum);
            if (lane == 0 && msum) {
                const uint32_t v = S.adj[rb + j] >> 1;
                if (out.vertex) atomicAdd(&O.pv[v], msum);
                if (peS) atomicAdd(&peS[rb + j], msum);  // edge w-v
            }
        }
        __syncwarp();
        // pairs: C(S,2) + C(A,2) to the endpoint and (summed) to the anchor;
        // the counters are reset as they are read
        const uint32_t first = __reduce_min_sync(FULL, wmin) >> 1;  // word index
        unsigned long long wsum = 0;
        for (uint32_t q = first + lane; q < HUB_WINDOW / 2; q += 32) {
            const uint32_t word = sm.win[q];
            if (!word) continue;
            sm.win[q] = 0;
            if (!out.vertex) continue;
#pragma unroll
            for (uint32_t h = 0; h < 2; h++) {
                const uint32_t c = (word >> (16 * h)) & 0xffffu;
                const unsigned long long b = c2(c & 0xffu) + c2(c >> 8);
                if (b) { atomicAdd(&S.pv[wb + 2 * q + h], b); wsum += b; }
            }
        }
        for (uint32_t i = lane; i < cap; i += 32) {
            const unsigned long long x = sm.tab[i];
            if (!x) continue;
            sm.tab[i] = 0ull;
            if (!out.vertex) continue;
            const uint32_t c = (uint32_t)x;
            const unsigned long long b = c2(c & 0xffffu) + c2(c >> 16);
            if (b) { atomicAdd(&S.pv[(uint32_t)(x >> 32) - 1u], b); wsum += b; }
        }
        wsum = warp_sum_u64(wsum);
        if (lane == 0 && wsum) atomicAdd(&S.pv[r], wsum);
        __syncwarp();
    }
}

// per-edge counts in the caller's edge order: an input edge (u, v) is the
// entry of v in u's U-side row and the entry of u in v's V-side row; its
// count is the sum of the two entries' counts
__global__ void k_pe_out(DevGraph G, const unsigned long long *peU,
                         const unsigned long long *peV, int64_t *out) {
    const SideCSR &U = G.side[0];
    const SideCSR &V = G.side[1];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < G.nE;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = G.nU;  // last u with rowptr[u] <= e
        while (hi - lo > 1) {
            const int64_t m = (lo + hi) >> 1;
            if (G.rowptr[m] <= e) lo = m; else hi = m;
        }
        const uint32_t ru = U.sr_of_id[lo];
        const uint32_t rv = V.sr_of_id[G.col[e]];
        const int64_t p = lower_bound_u32(U.adj, U.off[ru], U.off[ru + 1], rv << 1);
        const int64_t q = lower_bound_u32(V.adj, V.off[rv], V.off[rv + 1], ru << 1);
        out[e] = (int64_t)(peU[p] + peV[q]);
    }
}

// per-vertex counts from side-rank order to the caller's id order
__global__ void k_pv_out(SideCSR S, int64_t base, int64_t *out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < S.n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[base + S.id_of_sr[r]] = (int64_t)S.pv[r];
}

// grids of the three per-vertex kernels, once per device (any thread may
// count on any device)
struct PvCfg {
    int pv = 0, pvt = 0, pvw = 0;
};
constexpr int MAX_DEVICES = 64;
PvCfg g_pv_cfg[MAX_DEVICES];
std::once_flag g_pv_once[MAX_DEVICES];
constexpr size_t PVW_SMEM = (PVW_THREADS / 32) * sizeof(PvWarpSmem);
constexpr size_t PV_SMEM = sizeof(PvSmem<PV_THREADS, PV_DENSE_CAP>);
constexpr size_t PVT_SMEM = sizeof(PvSmem<PVT_THREADS, PVT_WORDS>);
auto *const k_pv_big = k_pv<PV_THREADS, PV_DENSE_CAP, false>;
auto *const k_pv_team = k_pv<PVT_THREADS, PVT_WORDS, true>;

template <typename K>
int pv_blocks(K kernel, int threads, size_t smem, int sms) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem);
    return std::max(1, b) * sms;
}

const PvCfg &pv_init() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        dev = 0;
    }
    std::call_once(g_pv_once[dev], [dev]() {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, dev);
        const int sms = prop.multiProcessorCount;
        PvCfg &c = g_pv_cfg[dev];
        c.pv = pv_blocks(k_pv_big, PV_THREADS, PV_SMEM, sms);
        c.pvt = pv_blocks(k_pv_team, PVT_THREADS, PVT_SMEM, sms);
        c.pvw = pv_blocks(k_pv_warp, PVW_THREADS, PVW_SMEM, sms);
    });
    return g_pv_cfg[dev];
}

// the three per-vertex walks: warp-class, team-class, then dense and
// CTA-hash anchors (each kernel drains its own job cursor)
void launch_pv_kernels(const DevGraph &g, const PvOut &o, cudaStream_t s) {
    const PvCfg &c = pv_init();
    cudaMemsetAsync(&g.scratch->job_next[JOB_PV_TEAM], 0, 4, s);
    cudaMemsetAsync(&g.scratch->job_next[JOB_PER_VERTEX], 0, 4, s);
    k_pv_warp<<<c.pvw, PVW_THREADS, PVW_SMEM, s>>>(g, o); note_launch();
    k_pv_team<<<c.pvt, PVT_THREADS, PVT_SMEM, s>>>(g, o); note_launch();
    k_pv_big<<<c.pv, PV_THREADS, PV_SMEM, s>>>(g, o); note_launch();
}

}  // namespace

void launch_per_edge(const DevGraph &g, int64_t *out_dev, unsigned long long *pe_ws,
                     cudaStream_t s) {
    pv_init();
    if (g.nE == 0) return;
    unsigned long long *peU = pe_ws, *peV = pe_ws + g.nE;
    cudaMemsetAsync(pe_ws, 0, (size_t)g.nE * 16, s);
    PvOut o{0, {peU, peV}};
    launch_pv_kernels(g, o, s);
    const int64_t blocks = std::min<int64_t>((g.nE + 255) / 256, 16384);
    k_pe_out<<<(unsigned)blocks, 256, 0, s>>>(g, peU, peV, out_dev); note_launch();
}

void launch_per_vertex(const DevGraph &g, int64_t *out_dev, cudaStream_t s) {
    pv_init();
    for (int sd = 0; sd < 2; sd++)
        if (g.side[sd].n > 0)
            cudaMemsetAsync(g.side[sd].pv, 0, (size_t)g.side[sd].n * 8, s);
    PvOut o{1, {nullptr, nullptr}};
    launch_pv_kernels(g, o, s);
    for (int sd = 0; sd < 2; sd++) {
        const int64_t n = g.side[sd].n;
        if (n == 0) continue;
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
        k_pv_out<<<(unsigned)blocks, 256, 0, s>>>(g.side[sd], sd ? g.nU : 0, out_dev); note_launch();
    }
}

}  // namespace bb
