// pervertex.cu - balanced butterflies containing each vertex (the quantity
// Algorithm 3 computes for one vertex), for every vertex at once, and
// containing each edge (the paper's edge-level extension), computed
// together with the counts in one set of launches.
//
// Each balanced butterfly is tallied at exactly one pair (w, u) of same-side
// vertices (w the anchor, u the higher-priority endpoint; see graph.cuh) and
// has two middles of the same wedge type. A pair with S symmetric and A
// asymmetric middles holds C(S,2) + C(A,2) balanced butterflies (Lemma 2):
// every one contains w and u, and a middle of type t lies in cnt_t - 1 of
// them (it pairs with each other middle of its type). Per anchor the
// kernels run
//   1. the count's tally pass (walk.cuh), which also gives the counts and,
//      summed over the anchor's wedges, the anchor's own balanced count;
//   2. a second walk over the same wedges reading the final tallies: each
//      wedge's cnt_t - 1, summed per middle by the walkers' segment sums;
//   3. a pass over the counters that adds each pair's C(S,2) + C(A,2) to
//      the endpoint and resets the counters.
//
// Per-edge counts come from the same second walk: a middle v of type t at
// pair (w, u) puts its cnt_t - 1 balanced butterflies on the edges w-v and
// v-u, accumulated per adjacency entry of each side (the entry of v in w's
// row and of u in v's row) and summed per input edge at the end.
//
// Dense anchors split over several CTAs take two launches: the parts tally
// and merge into the group's global counters (k_pv_dense), then every part
// copies the final counters and walks its middles again, and the first
// part scans the counters (k_pv_split). Wide anchors (degree above
// MAX_DEGREE, 32-bit tally fields) go to k_pv_wide.
#include <algorithm>
#include <mutex>
#include "edgerows.cuh"
#include "walk.cuh"

namespace bb {

namespace {

using namespace walk;

// What the kernels accumulate: per-vertex counts (into each side's pv
// array) and/or per-edge counts (into pe[side][position of the entry in
// that side's adjacency]; null when not wanted).
struct PvOut {
    int vertex;
    unsigned long long *pe[2];
};

// Per CTA of the warp class, the per-vertex sums of the top HUB_WINDOW
// ranks of each side (the hub windows: U side, then V side) in shared
// memory, u32 with the carry going to the global sum. The top ranks are
// endpoints and middles of most warp-class anchors, so their additions stay
// in shared memory and reach global memory once per CTA (hub_flush) instead
// of serialising on a few global addresses (measured: 25 ms against 13 ms
// for the warp class on the 2M x 500k graph). The larger classes have few
// anchors per CTA; there the shared arrays only cost occupancy.
constexpr size_t HUB_SUMS_BYTES = 2 * HUB_WINDOW * 4;

// The outputs of one anchor: its own side's per-vertex sums (anchor and
// endpoints) and adjacency (its middles), the middles' side's per-vertex
// sums, the per-entry sums of both sides (null when not wanted), and the
// CTA's hub-window sums of both sides with their windows' first ranks.
struct PvSides {
    const uint32_t *sadj;
    unsigned long long *spv, *opv;
    unsigned long long *peS, *peO;
    uint32_t *hubS, *hubO;
    uint32_t wbS, wbO;
};

__device__ __forceinline__ PvSides pv_sides(const DevGraph &G, const PvOut &out, uint32_t anchor,
                                            uint32_t *hub) {
    const bool v = anchor & 1u;
    PvSides p;
    p.sadj = v ? G.side[1].adj : G.side[0].adj;
    p.spv = out.vertex ? (v ? G.side[1].pv : G.side[0].pv) : nullptr;
    p.opv = out.vertex ? (v ? G.side[0].pv : G.side[1].pv) : nullptr;
    p.peS = v ? out.pe[1] : out.pe[0];
    p.peO = v ? out.pe[0] : out.pe[1];
    p.hubS = hub ? hub + (v ? HUB_WINDOW : 0u) : nullptr;
    p.hubO = hub ? hub + (v ? 0u : HUB_WINDOW) : nullptr;
    p.wbS = window_base(v ? G.side[1].n : G.side[0].n);
    p.wbO = window_base(v ? G.side[0].n : G.side[1].n);
    return p;
}

// slot of hub-window counter index i (rank mod HUB_WINDOW) in a side's
// hub sums: even indexes first, then odd ones, so that lanes reading
// consecutive words of a 16-bit counter window add to consecutive slots
__device__ __forceinline__ uint32_t hub_slot(uint32_t i) {
    return (i & 1u) * (HUB_WINDOW / 2) + (i >> 1);
}

// Hub slots hold twice their vertices' sums (mod 2^32): the warp class adds
// its endpoints' pair counts wedge by wedge, and the wedges of a pair with
// final tallies S, A add (S - 1) S + (A - 1) A = 2 (C(S,2) + C(A,2)).
// hub_add2 adds d (twice a sum) to the slot of rank u; a carry past 2^32
// is 2^31 of the vertex's sum and goes to the global sum.
__device__ __forceinline__ void hub_add2(uint32_t *hub, unsigned long long *pv, uint32_t slot,
                                         uint32_t u, uint32_t d) {
    const uint32_t old = atomicAdd(&hub[slot], d);
    if (old + d < old) atomicAdd(&pv[u], 1ull << 31);
}

// adds b to the per-vertex sum of rank u of a side (pv; its CTA hub sums
// hub or null, window base wb)
__device__ __forceinline__ void pv_add(unsigned long long *pv, uint32_t *hub, uint32_t wb,
                                       uint32_t u, unsigned long long b) {
    if (hub && u >= wb && (b >> 31) == 0)
        hub_add2(hub, pv, hub_slot(u & (HUB_WINDOW - 1)), u, (uint32_t)b << 1);
    else
        atomicAdd(&pv[u], b);
}

// adds a CTA's hub-window sums to the global per-vertex sums
template <int TS>
__device__ __forceinline__ void hub_flush(const DevGraph &G, const uint32_t *hub) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 2 * HUB_WINDOW; i += TS) {
        const uint32_t v = hub[i];
        if (!v) continue;
        const bool sv = i >= HUB_WINDOW;
        unsigned long long *pv = sv ? G.side[1].pv : G.side[0].pv;
        const uint32_t wb = window_base(sv ? G.side[1].n : G.side[0].n);
        const uint32_t j = i & (HUB_WINDOW - 1);  // slot -> counter index
        const uint32_t ci = ((j & (HUB_WINDOW / 2 - 1)) << 1) | (j / (HUB_WINDOW / 2));
        atomicAdd(&pv[window_rank(ci, wb)], (unsigned long long)(v >> 1));
    }
}

template <int TS>
__device__ __forceinline__ void hub_zero(uint32_t *hub) {
    for (uint32_t i = threadIdx.x; i < 2 * HUB_WINDOW; i += TS) hub[i] = 0u;
}

// a wedge whose middle has k other middles of its type at the pair: the
// edge middle-endpoint (entry p of the middle's row) lies in k balanced
// butterflies there; k is the walker's value for the middle's sum
__device__ __forceinline__ uint32_t pv_entry(const PvSides &P, uint32_t p, uint32_t k) {
    if (P.peO && k) atomicAdd(&P.peO[p], (unsigned long long)k);
    return k;
}

// middle j of the anchor's row (row start rb) lies in s balanced
// butterflies at this anchor, and so does the edge anchor-middle
__device__ __forceinline__ void pv_middle(const PvSides &P, int64_t rb, uint32_t j,
                                          unsigned long long s) {
    if (!s) return;
    if (P.opv) pv_add(P.opv, P.hubO, P.wbO, P.sadj[rb + j] >> 1, s);
    if (P.peS) atomicAdd(&P.peS[rb + j], s);
}

// the endpoint u of a pair with b = C(S,2) + C(A,2) lies in b of them
__device__ __forceinline__ void pv_pair(const PvSides &P, uint32_t u, unsigned long long b) {
    if (b && P.spv) pv_add(P.spv, P.hubS, P.wbS, u, b);
}

__device__ __forceinline__ unsigned long long pair_b16(uint32_t c) {
    return c2(c & 0xffffu) + c2(c >> 16);
}

// endpoints of a hash table's pairs (S | A << 16 in the low half, endpoint
// + 1 in the high half), slots reset as they are read, by TS threads
template <int TS>
__device__ __forceinline__ void pv_table_pairs(const PvSides &P, unsigned long long *tab,
                                               uint32_t cap, int t) {
    for (uint32_t i = t; i < cap; i += TS) {
        const unsigned long long x = tab[i];
        if (!x) continue;
        tab[i] = 0ull;
        pv_pair(P, (uint32_t)(x >> 32) - 1u, pair_b16((uint32_t)x));
    }
}

// ------------------------------------------------------------ warp class
// One anchor per warp with the count's layout (WarpSmem: the hub window in
// 16-bit counters of two bytes S | A << 8, the hash below it) plus the
// second walk's segment sums.
struct alignas(16) PvWarpSmem {
    WarpSmem w;
    uint32_t acc[64];
};
static_assert(offsetof(PvWarpSmem, w) == 0 && sizeof(PvWarpSmem) % 16 == 0,
              "per-warp copies back to back");

__device__ __forceinline__ void pv_warp_anchor(const DevGraph &G, PvWarpSmem &pw, uint32_t *hub,
                                               const AnchorRec &rec, const PvOut &out,
                                               unsigned lane, unsigned long long &bal,
                                               unsigned long long &tot) {
    WarpSmem &sm = pw.w;
    uint32_t *err = &G.scratch->err;
    const Anchor A = load_anchor(G, rec);
    const PvSides P = pv_sides(G, out, rec.anchor, out.vertex ? hub : nullptr);
    uint32_t own = 0, other = 0;
    const WarpTab tb = warp_tally(G, sm, rec, A, lane, own, other);
    bal += own;
    tot += (unsigned long long)own + other;
    __syncwarp();
    // second walk: a wedge of type t reads its pair's final tally cnt_t
    const uint32_t mask = tb.cap - 1, shift = tb.shift;
    const unsigned char *winb = reinterpret_cast<const unsigned char *>(sm.win);
    auto low = [&](uint32_t x, uint32_t sw, uint32_t p) -> uint32_t {
        const uint32_t c = hash_find(sm.tab, shift, mask, (x >> 1) + 1, err);
        const uint32_t ct = ((x ^ sw) & 1u) ? c >> 16 : c & 0xffffu;
        return pv_entry(P, p, ct ? ct - 1u : 0u);
    };
    // the tally's byte: bit 1 of x picks the half, the sign xor bit 0 the
    // type; the wedge's cnt_t - 1 also goes to its endpoint's hub slot
    // (twice the pair's count over the pair's wedges)
    auto hubw = [&](uint32_t x, uint32_t vb, uint32_t sw, uint32_t p) -> uint32_t {
        const uint32_t ct = winb[(x & (2u * HUB_WINDOW - 4u)) | ((x ^ sw) & 3u)];
        const uint32_t k = vb ? ct - 1u : 0u;
        if (P.hubS && k) hub_add2(P.hubS, P.spv, hub_slot((x >> 1) & (HUB_WINDOW - 1)), x >> 1, k);
        return pv_entry(P, p, k);
    };
    auto mid = [&](uint32_t j, unsigned long long s) { pv_middle(P, A.rb, j, s); };
    if (tb.hub) {
        warp_rounds<true>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, lane, HubSeg{},
                          [&](const uint4 &v, uint32_t vm, uint32_t sw, uint32_t p) -> uint32_t {
                              return hubw(v.x, vm & 1u, sw, p) +
                                     hubw(v.y, (vm >> 1) & 1u, sw, p + 1) +
                                     hubw(v.z, (vm >> 2) & 1u, sw, p + 2) +
                                     hubw(v.w, vm >> 3, sw, p + 3);
                          },
                          LowSeg{}, low, pw.acc, mid);
    } else {
        warp_rounds<true>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, lane,
                          [](const uint4 &, long long &st, uint32_t &len) { st = 0; len = 0; },
                          [](const uint4 &, uint32_t, uint32_t, uint32_t) -> uint32_t { return 0u; },
                          FullSeg{}, low, pw.acc, mid);
    }
    // endpoints: the hub window's went to the hub slots wedge by wedge, so
    // its counters are only reset; the hash's C(S,2) + C(A,2) per pair
    if (tb.hub) {
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = lane; q < HUB_WINDOW / 8; q += 32) w4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    pv_table_pairs<32>(P, sm.tab, tb.cap, (int)lane);
    // the anchor lies in all its balanced butterflies: the sum over its
    // wedges of their own tallies' previous values (below 2^32 per anchor)
    if (P.spv) {
        const uint32_t wsum = __reduce_add_sync(FULL, own);
        if (lane == 0 && wsum) atomicAdd(&P.spv[A.r], (unsigned long long)wsum);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(WARP_THREADS, 3) k_pv_warp(DevGraph G, PvOut out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned lane = lane_id();
    PvWarpSmem &pw =
        reinterpret_cast<PvWarpSmem &>(warp_smem_init(smem_raw, lane, sizeof(PvWarpSmem)));
    pw.acc[lane] = 0u;
    pw.acc[32 + lane] = 0u;
    uint32_t *hub = reinterpret_cast<uint32_t *>(smem_raw + (WARP_THREADS / 32) * sizeof(PvWarpSmem));
    hub_zero<WARP_THREADS>(hub);
    __syncthreads();
    const uint32_t n = G.ctr[CTR_WARP];
    const uint32_t gw = (blockIdx.x * WARP_THREADS + threadIdx.x) >> 5;
    const uint32_t GW = (gridDim.x * WARP_THREADS) >> 5;
    unsigned long long bal = 0, tot = 0;
    AnchorRec cur;
    if (gw < n) cur = G.warp_list[gw];
    for (uint32_t idx = gw; idx < n; idx += GW) {
        AnchorRec nxt;
        if (idx + GW < n) nxt = G.warp_list[idx + GW];
        pv_warp_anchor(G, pw, hub, cur, out, lane, bal, tot);
        spill_if_large(G.scratch, bal, tot);
        cur = nxt;
    }
    flush_warp(G.scratch, bal, tot);
    if (out.vertex) hub_flush<WARP_THREADS>(G, hub);
}

// ------------------------------------------------- team and CTA-hash classes
template <int TS, uint32_t HCAP>
struct alignas(16) PvHybSmem {
    HybSmem<TS, HCAP> h;
    unsigned long long acc[TS];
};

template <int TS, uint32_t HCAP>
__device__ __forceinline__ void pv_hybrid_anchor(const DevGraph &G, PvHybSmem<TS, HCAP> &ps,
                                                 const AnchorRec &rec, const PvOut &out,
                                                 unsigned long long &bal,
                                                 unsigned long long &tot) {
    HybSmem<TS, HCAP> &sm = ps.h;
    const int t = threadIdx.x;
    uint32_t *err = &G.scratch->err;
    const Anchor A = load_anchor(G, rec);
    const PvSides P = pv_sides(G, out, rec.anchor, nullptr);
    unsigned long long ab = 0, at = 0;  // this anchor's part of the counts
    const HybTab tb = hybrid_tally<TS, HCAP, false>(G, sm, A, ab, at);
    bal += ab;
    tot += at;
    __syncthreads();
    auto noflush = []() {};
    auto mid = [&](uint32_t j, unsigned long long s) { pv_middle(P, A.rb, j, s); };
    if (tb.hub)
        quad_walk<TS, HYBRID_QUADS<TS>, true, true>(
            A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, SUM_SPAN, HubSeg{},
            [&](uint32_t x, uint32_t vb, uint32_t sw, uint32_t p) -> uint32_t {
                const uint32_t c = sm.win[(x >> 1) & (HUB_WINDOW - 1)];
                const uint32_t ct = (c >> (((x ^ sw) & 1u) << 4)) & 0xffffu;
                return pv_entry(P, p, vb ? ct - 1u : 0u);
            },
            noflush, ps.acc, mid);
    if (tb.cap) {
        const uint32_t mask = tb.cap - 1, shift = tb.shift;
        wedge_walk<TS, 2, true>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, 4 * SUM_SPAN, LowSeg{},
                                [&](uint32_t x, uint32_t sw, uint32_t p) -> uint32_t {
                                    const uint32_t c =
                                        hash_find(sm.tab, shift, mask, (x >> 1) + 1, err);
                                    const uint32_t ct = ((x ^ sw) & 1u) ? c >> 16 : c & 0xffffu;
                                    return pv_entry(P, p, ct ? ct - 1u : 0u);
                                },
                                noflush, ps.acc, mid);
    }
    __syncthreads();
    if (tb.hub) {
        const uint32_t wb = window_base(A.ns);
        for (uint32_t i = t; i < HUB_WINDOW; i += TS) {
            const uint32_t c = sm.win[i];
            if (!c) continue;
            sm.win[i] = 0u;
            pv_pair(P, window_rank(i, wb), pair_b16(c));
        }
    }
    pv_table_pairs<TS>(P, sm.tab, tb.cap, t);
    if (P.spv) {
        block_sum2<TS>(ab, at);
        if (t == 0 && ab) atomicAdd(&P.spv[A.r], ab);
    }
}

template <int TS, uint32_t HCAP, int CTR, int CLS>
__device__ __forceinline__ void pv_hybrid_body(const DevGraph &G, const AnchorRec *list,
                                               const PvOut &out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = PvHybSmem<TS, HCAP>;
    static_assert(offsetof(Smem, h) == 0, "hybrid counters first");
    hybrid_smem_init<TS, HCAP>(smem_raw);
    Smem &ps = *reinterpret_cast<Smem *>(smem_raw);
    ps.acc[threadIdx.x] = 0ull;
    const uint32_t n = G.ctr[CTR];
    unsigned long long bal = 0, tot = 0;
    for (;;) {
        if (threadIdx.x == 0) ps.h.job = atomicAdd(&G.scratch->job_next[CLS], 1u);
        __syncthreads();
        const uint32_t jid = ps.h.job;
        __syncthreads();
        if (jid >= n) break;
        pv_hybrid_anchor<TS, HCAP>(G, ps, list[jid], out, bal, tot);
        spill_if_large(G.scratch, bal, tot);
    }
    block_sum2<TS>(bal, tot);
    if (threadIdx.x == 0) acc_add(G.scratch, bal, tot);
}

__global__ void __launch_bounds__(TEAM_THREADS) k_pv_team(DevGraph G, PvOut out) {
    pv_hybrid_body<TEAM_THREADS, TEAM_CAP, CTR_TEAM, CLS_TEAM>(G, G.team_list, out);
}

__global__ void __launch_bounds__(CTAH_THREADS) k_pv_ctah(DevGraph G, PvOut out) {
    pv_hybrid_body<CTAH_THREADS, CTAH_CAP, CTR_CTAH, CLS_CTAH>(G, G.ctah_list, out);
}

// ------------------------------------------------------------ dense class
// Dense counters (S | A << 16) over the anchor's endpoint range, walked in
// windows of DENSE_CAP endpoints when longer; u64 counters (S | A << 32)
// over half the range for wide anchors.
// acc: the second walk's per-middle sums. A middle's sum over one window
// (or one split anchor) is below DENSE_CAP wedges times the degree, which
// fits 32 bits; the u32 sums keep three CTAs per SM.
struct alignas(16) PvDenseSmem {
    uint32_t cnt[DENSE_CAP];
    WalkSmem<DENSE_THREADS> walk;
    uint32_t acc[DENSE_THREADS];
    uint32_t job, last;
};
static_assert((unsigned long long)DENSE_CAP * MAX_DEGREE < (1ull << 32), "u32 middle sums");

// the anchor of a dense job (its row start from the side's offsets)
__device__ __forceinline__ Anchor dense_anchor(const DevGraph &G, uint32_t anchor) {
    AnchorRec rec;
    rec.anchor = anchor;
    const int64_t *off = (anchor & 1u) ? G.side[1].off : G.side[0].off;
    rec.rb = (uint32_t)off[anchor >> 1];
    rec.deg = 0;
    rec.W = 0;
    rec.wnh = 0;
    return load_anchor(G, rec);
}

// the tally of dense counters over endpoints [e0, e0 + DENSE_CAP) by the
// middles [m0, m1); adds the wedges' previous tallies to ab (own) and at
// (both)
template <typename Seg>
__device__ __forceinline__ void dense_tally(PvDenseSmem &sm, const Anchor &A, uint32_t m0,
                                            uint32_t m1, uint32_t e0, Seg &&seg,
                                            unsigned long long &ab, unsigned long long &at) {
    uint32_t b32 = 0, t32 = 0;
    team_rounds<DENSE_THREADS, true>(
        A.smd, A.oadj, A.rb, m0, m1, sm.walk, threadIdx.x, SUM_SPAN, seg,
        [&](uint32_t x, uint32_t vb, uint32_t sw) {
            const uint32_t asym = (x ^ sw) & 1u;
            const uint32_t idx = ((x >> 1) - e0) & (DENSE_CAP - 1);
            const uint32_t old = atomicAdd(&sm.cnt[idx], vb << (asym << 4));
            b32 = __dp2a_lo(old, vb << (asym << 3), b32);
            t32 = __dp2a_lo(old, vb * 0x0101u, t32);
        },
        [&]() {
            ab += b32;
            at += t32;
            b32 = t32 = 0;
        });
}

// the second walk of the middles [m0, m1) over final dense counters
template <typename Seg>
__device__ __forceinline__ void dense_read(PvDenseSmem &sm, const Anchor &A, const PvSides &P,
                                           uint32_t m0, uint32_t m1, uint32_t e0, Seg &&seg) {
    team_rounds<DENSE_THREADS, true, true>(
        A.smd, A.oadj, A.rb, m0, m1, sm.walk, threadIdx.x, SUM_SPAN, seg,
        [&](uint32_t x, uint32_t vb, uint32_t sw, uint32_t p) -> uint32_t {
            const uint32_t idx = ((x >> 1) - e0) & (DENSE_CAP - 1);
            const uint32_t ct = (sm.cnt[idx] >> (((x ^ sw) & 1u) << 4)) & 0xffffu;
            return pv_entry(P, p, vb ? ct - 1u : 0u);
        },
        []() {}, sm.acc, [&](uint32_t j, unsigned long long s) { pv_middle(P, A.rb, j, s); });
}

// endpoints [e0, e0 + len) of dense counters (adds the pairs' balanced
// butterflies to ab when asked)
__device__ __forceinline__ void dense_pairs(const PvDenseSmem &sm, const PvSides &P, uint32_t e0,
                                            uint32_t len) {
    if (!P.spv) return;
    for (uint32_t i = threadIdx.x; i < len; i += DENSE_THREADS)
        pv_pair(P, e0 + i, pair_b16(sm.cnt[i]));
}

// A dense anchor walked whole by one CTA: per window of endpoints, tally,
// second walk, endpoints.
__device__ __forceinline__ void pv_dense_job(const DevGraph &G, PvDenseSmem &sm, const DenseJob &J,
                                             const PvOut &out, unsigned long long &bal,
                                             unsigned long long &tot) {
    const int t = threadIdx.x;
    const Anchor A = dense_anchor(G, J.anchor);
    const PvSides P = pv_sides(G, out, J.anchor, nullptr);
    const uint32_t e_lo = A.r + 1, e_hi = (uint32_t)A.ns;
    const bool windows = (e_hi - e_lo) > DENSE_CAP;
    unsigned long long ab = 0, at = 0;
    for (uint32_t e0 = e_lo; e0 < e_hi; e0 += DENSE_CAP) {
        const uint32_t e1 = e_hi - e0 > DENSE_CAP ? e0 + DENSE_CAP : e_hi;
        const uint32_t len = e1 - e0;
        for (uint32_t i = t; i < len; i += DENSE_THREADS) sm.cnt[i] = 0;
        __syncthreads();
        if (windows) {
            auto clipped = [&](const uint4 &d, long long &st, uint32_t &l) {
                const long long s0 = lower_bound_u32(A.oadj, d.x, d.z, e0 << 1);
                st = s0;
                l = (uint32_t)(lower_bound_u32(A.oadj, s0, d.z, e1 << 1) - s0);
            };
            dense_tally(sm, A, J.m0, J.m1, e0, clipped, ab, at);
            __syncthreads();
            dense_read(sm, A, P, J.m0, J.m1, e0, clipped);
        } else {
            dense_tally(sm, A, J.m0, J.m1, e0, FullSeg{}, ab, at);
            __syncthreads();
            dense_read(sm, A, P, J.m0, J.m1, e0, FullSeg{});
        }
        __syncthreads();
        dense_pairs(sm, P, e0, len);
        __syncthreads();  // the next window rewrites the counters
    }
    bal += ab;
    tot += at;
    if (P.spv) {
        block_sum2<DENSE_THREADS>(ab, at);
        if (t == 0 && ab) atomicAdd(&P.spv[A.r], ab);
    }
}

// One part of a split anchor, first launch: tally its middles and merge
// into the group's global counters (a count p added to c already there
// closes c*p new pairs across parts); the merged counters stay for the
// second launch.
__device__ __forceinline__ void pv_split_tally(const DevGraph &G, PvDenseSmem &sm,
                                               const DenseJob &J, unsigned long long &bal,
                                               unsigned long long &tot) {
    const int t = threadIdx.x;
    const Anchor A = dense_anchor(G, J.anchor);
    const SplitGroup grp = G.groups[J.group];
    const uint32_t e0 = A.r + 1, len = grp.len;
    for (uint32_t i = t; i < len; i += DENSE_THREADS) sm.cnt[i] = 0;
    __syncthreads();
    dense_tally(sm, A, J.m0, J.m1, e0, FullSeg{}, bal, tot);
    __syncthreads();
    uint32_t *part = G.gpart + grp.goff;
    for (uint32_t i = t; i < len; i += DENSE_THREADS) {
        const uint32_t p = sm.cnt[i];
        if (p) {
            const uint32_t c = atomicAdd(&part[i], p);
            const unsigned long long cS = c & 0xffffu, cA = c >> 16;
            const unsigned long long pS = p & 0xffffu, pA = p >> 16;
            bal += cS * pS + cA * pA;
            tot += (cS + cA) * (pS + pA);
        }
    }
    __syncthreads();  // the next job rewrites the counters
}

__global__ void __launch_bounds__(DENSE_THREADS, 3) k_pv_dense(DevGraph G, PvOut out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PvDenseSmem &sm = *reinterpret_cast<PvDenseSmem *>(smem_raw);
    sm.acc[threadIdx.x] = 0u;
    const uint32_t njobs = G.ctr[CTR_DENSE];
    unsigned long long bal = 0, tot = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(&G.scratch->job_next[CLS_DENSE], 1u);
        __syncthreads();
        const uint32_t jid = sm.job;
        __syncthreads();
        if (jid >= njobs) break;
        const DenseJob J = G.dense_jobs[jid];
        if (J.group == NO_GROUP) pv_dense_job(G, sm, J, out, bal, tot);
        else if (J.group != WIDE_JOB) pv_split_tally(G, sm, J, bal, tot);
        spill_if_large(G.scratch, bal, tot);
    }
    flush_warp(G.scratch, bal, tot);
}

// thread 0 takes the next job of the dense list whose group passes keep()
// from cursor `which` (njobs when none is left)
template <typename Keep>
__device__ __forceinline__ uint32_t next_dense_job(const DevGraph &G, PvDenseSmem &sm, int which,
                                                   uint32_t njobs, Keep &&keep) {
    if (threadIdx.x == 0) {
        uint32_t j = atomicAdd(&G.scratch->job_next[which], 1u);
        while (j < njobs && !keep(G.dense_jobs[j].group))
            j = atomicAdd(&G.scratch->job_next[which], 1u);
        sm.job = j;
    }
    __syncthreads();
    const uint32_t jid = sm.job;
    __syncthreads();
    return jid;
}

// Second launch for split parts: copy the group's final counters, release
// them (the last part to copy resets them for the next count), walk this
// part's middles; the first part (m0 = 0) adds the endpoints' and the
// anchor's sums.
__global__ void __launch_bounds__(DENSE_THREADS, 3) k_pv_split(DevGraph G, PvOut out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PvDenseSmem &sm = *reinterpret_cast<PvDenseSmem *>(smem_raw);
    const int t = threadIdx.x;
    sm.acc[t] = 0u;
    const uint32_t njobs = G.ctr[CTR_DENSE];
    for (;;) {
        const uint32_t jid = next_dense_job(G, sm, JOB_PV_SPLIT, njobs, [](uint32_t g) {
            return g != NO_GROUP && g != WIDE_JOB;
        });
        if (jid >= njobs) break;
        const DenseJob J = G.dense_jobs[jid];
        const SplitGroup grp = G.groups[J.group];
        const Anchor A = dense_anchor(G, J.anchor);
        const PvSides P = pv_sides(G, out, J.anchor, nullptr);
        const uint32_t e0 = A.r + 1, len = grp.len;
        uint32_t *part = G.gpart + grp.goff;
        for (uint32_t i = t; i < len; i += DENSE_THREADS) sm.cnt[i] = part[i];
        __threadfence();
        __syncthreads();
        if (t == 0) sm.last = atomicAdd(&G.gdone[J.group], 1u) == grp.parts - 1 ? 1u : 0u;
        __syncthreads();
        if (sm.last) {  // every part has its copy
            for (uint32_t i = t; i < len; i += DENSE_THREADS) part[i] = 0;
            if (t == 0) G.gdone[J.group] = 0;
        }
        dense_read(sm, A, P, J.m0, J.m1, e0, FullSeg{});
        __syncthreads();
        if (J.m0 == 0 && P.spv) {
            unsigned long long ab = 0, at = 0;
            for (uint32_t i = t; i < len; i += DENSE_THREADS) {
                const unsigned long long b = pair_b16(sm.cnt[i]);
                pv_pair(P, e0 + i, b);
                ab += b;
            }
            block_sum2<DENSE_THREADS>(ab, at);
            if (t == 0 && ab) atomicAdd(&P.spv[A.r], ab);
        }
        __syncthreads();  // the next job rewrites the counters
    }
}

// Wide anchors (degree above MAX_DEGREE): u64 counters (S | A << 32) over
// windows of DENSE_CAP / 2 endpoints; the second walk takes one warp per
// middle (these anchors are few) and sums in 64 bits.
__global__ void __launch_bounds__(DENSE_THREADS) k_pv_wide(DevGraph G, PvOut out) {
    constexpr uint32_t CAP = DENSE_CAP / 2;
    constexpr uint32_t NW = DENSE_THREADS / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PvDenseSmem &sm = *reinterpret_cast<PvDenseSmem *>(smem_raw);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(sm.cnt);
    const int t = threadIdx.x;
    const uint32_t lane = (uint32_t)t & 31u, warp = (uint32_t)t >> 5;
    const uint32_t njobs = G.ctr[CTR_DENSE];
    unsigned long long bal = 0, tot = 0;
    for (;;) {
        const uint32_t jid = next_dense_job(G, sm, JOB_WIDE, njobs,
                                            [](uint32_t g) { return g == WIDE_JOB; });
        if (jid >= njobs) break;
        const DenseJob J = G.dense_jobs[jid];
        const Anchor A = dense_anchor(G, J.anchor);
        const PvSides P = pv_sides(G, out, J.anchor, nullptr);
        const uint32_t e_lo = A.r + 1, e_hi = (uint32_t)A.ns;
        const bool windows = (e_hi - e_lo) > CAP;
        unsigned long long ab = 0, at = 0;
        unsigned long long anc = 0;  // this thread's part of the anchor's balanced count
        for (uint32_t e0 = e_lo; e0 < e_hi; e0 += CAP) {
            const uint32_t e1 = e_hi - e0 > CAP ? e0 + CAP : e_hi;
            const uint32_t len = e1 - e0;
            for (uint32_t i = t; i < len; i += DENSE_THREADS) cnt[i] = 0ull;
            __syncthreads();
            auto seg = [&](const uint4 &d, long long &st, uint32_t &l) {
                if (windows) {
                    const long long s0 = lower_bound_u32(A.oadj, d.x, d.z, e0 << 1);
                    st = s0;
                    l = (uint32_t)(lower_bound_u32(A.oadj, s0, d.z, e1 << 1) - s0);
                } else {
                    st = d.x;
                    l = d.z - d.x;
                }
            };
            team_rounds<DENSE_THREADS, true>(
                A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t, 1024, seg,
                [&](uint32_t x, uint32_t vb, uint32_t sw) {
                    const uint32_t asym = (x ^ sw) & 1u;
                    const uint32_t idx = ((x >> 1) - e0) & (CAP - 1);
                    const unsigned long long old =
                        atomicAdd(&cnt[idx], (unsigned long long)vb << (asym << 5));
                    const unsigned long long oS = old & 0xffffffffull, oA = old >> 32;
                    if (vb) {
                        ab += asym ? oA : oS;
                        at += oS + oA;
                    }
                },
                [&]() {
                    bal += ab;
                    tot += at;
                    anc += ab;
                    ab = at = 0;
                    spill_if_large(G.scratch, bal, tot);
                });
            __syncthreads();
            for (uint32_t j = J.m0 + warp; j < J.m1; j += NW) {
                const uint4 d = A.smd[A.rb + j];
                long long st;
                uint32_t l;
                seg(d, st, l);
                unsigned long long ms = 0;
                for (uint32_t p = (uint32_t)st + lane; p < (uint32_t)st + l; p += 32) {
                    const uint32_t x = A.oadj[p];
                    const unsigned long long c = cnt[((x >> 1) - e0) & (CAP - 1)];
                    const unsigned long long ct = ((x ^ d.w) & 1u) ? c >> 32 : c & 0xffffffffull;
                    const unsigned long long k = ct ? ct - 1 : 0;
                    ms += k;
                    if (P.peO && k) atomicAdd(&P.peO[p], k);
                }
                ms = warp_sum_u64(ms);
                if (lane == 0) pv_middle(P, A.rb, j, ms);
            }
            __syncthreads();
            if (P.spv)
                for (uint32_t i = t; i < len; i += DENSE_THREADS) {
                    const unsigned long long c = cnt[i];
                    pv_pair(P, e0 + i, c2(c & 0xffffffffull) + c2(c >> 32));
                }
            __syncthreads();  // the next window rewrites the counters
        }
        if (P.spv) {
            unsigned long long unused = 0;
            block_sum2<DENSE_THREADS>(anc, unused);
            if (t == 0 && anc) atomicAdd(&P.spv[A.r], anc);
        }
    }
    flush_warp(G.scratch, bal, tot);
}

// per-edge counts in the caller's edge order: an input edge (u, v) is the
// entry of v in u's U-side row and the entry of u in v's V-side row; its
// count is the sum of the two entries' counts. A block takes consecutive
// input edges per step and finds their rows without a search per edge.
__global__ void __launch_bounds__(edgerows::THREADS) k_pe_out(DevGraph G,
                                                              const unsigned long long *peU,
                                                              const unsigned long long *peV,
                                                              int64_t *out) {
    __shared__ edgerows::Smem er;
    const int t = threadIdx.x;
    const int64_t nE = G.nE;
    for (int64_t e0 = blockIdx.x * (int64_t)edgerows::EDGES; e0 < nE;
         e0 += (int64_t)gridDim.x * edgerows::EDGES) {
        const int64_t e1 = nE - e0 > edgerows::EDGES ? e0 + edgerows::EDGES : nE;
        const int64_t u0 = edgerows::step_rows(G.rowptr, G.nU, e0, e1, er);
        for (int64_t e = e0 + t; e < e1; e += edgerows::THREADS) {
            const uint32_t ru = G.side[0].sr_of_id[u0 + er.srow[e - e0] - 1];
            const uint32_t rv = G.side[1].sr_of_id[G.col[e]];
            const int64_t p = lower_bound_u32(G.side[0].adj, G.side[0].off[ru], G.side[0].off[ru + 1],
                                              rv << 1);
            const int64_t q = lower_bound_u32(G.side[1].adj, G.side[1].off[rv], G.side[1].off[rv + 1],
                                              ru << 1);
            out[e] = (int64_t)(peU[p] + peV[q]);
        }
        __syncthreads();  // the next step rewrites the shared rows
    }
}

// per-vertex counts from side-rank order to the caller's id order
__global__ void k_pv_out(SideCSR S, int64_t base, int64_t *out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < S.n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[base + S.id_of_sr[r]] = (int64_t)S.pv[r];
}

// grids of the per-vertex kernels, once per device (any thread may count
// on any device)
struct PvCfg {
    int warp = 0, team = 0, ctah = 0, dense = 0, sms = 0;
};
constexpr int MAX_DEVICES = 64;
PvCfg g_pv_cfg[MAX_DEVICES];
std::once_flag g_pv_once[MAX_DEVICES];
constexpr size_t PVW_SMEM = (WARP_THREADS / 32) * sizeof(PvWarpSmem) + HUB_SUMS_BYTES;
constexpr size_t PVT_SMEM = sizeof(PvHybSmem<TEAM_THREADS, TEAM_CAP>);
constexpr size_t PVC_SMEM = sizeof(PvHybSmem<CTAH_THREADS, CTAH_CAP>);
constexpr size_t PVD_SMEM = sizeof(PvDenseSmem);

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
        c.sms = sms;
        c.warp = pv_blocks(k_pv_warp, WARP_THREADS, PVW_SMEM, sms);
        c.team = pv_blocks(k_pv_team, TEAM_THREADS, PVT_SMEM, sms);
        c.ctah = pv_blocks(k_pv_ctah, CTAH_THREADS, PVC_SMEM, sms);
        c.dense = pv_blocks(k_pv_dense, DENSE_THREADS, PVD_SMEM, sms);
        pv_blocks(k_pv_split, DENSE_THREADS, PVD_SMEM, sms);  // shared-memory opt-ins
        pv_blocks(k_pv_wide, DENSE_THREADS, PVD_SMEM, sms);
    });
    return g_pv_cfg[dev];
}

// The count with the per-vertex or per-edge walks, in the count's order
// (dense, CTA-hash, team, warp; events as launch_count records them).
void launch_pv_kernels(const DevGraph &g, const PvOut &o, cudaStream_t s, cudaEvent_t *ev) {
    const PvCfg &c = pv_init();
    cudaMemsetAsync(g.scratch, 0, sizeof(CountScratch), s);
    if (ev) record_timing_event(ev[0], s);
    k_pv_dense<<<c.dense, DENSE_THREADS, PVD_SMEM, s>>>(g, o); note_launch();
    k_pv_split<<<c.dense, DENSE_THREADS, PVD_SMEM, s>>>(g, o); note_launch();
    if (g.h_maxdeg > MAX_DEGREE) { k_pv_wide<<<c.sms, DENSE_THREADS, PVD_SMEM, s>>>(g, o); note_launch(); }
    if (ev) record_timing_event(ev[1], s);
    k_pv_ctah<<<c.ctah, CTAH_THREADS, PVC_SMEM, s>>>(g, o); note_launch();
    if (ev) record_timing_event(ev[2], s);
    k_pv_team<<<c.team, TEAM_THREADS, PVT_SMEM, s>>>(g, o); note_launch();
    if (ev) record_timing_event(ev[3], s);
    k_pv_warp<<<c.warp, WARP_THREADS, PVW_SMEM, s>>>(g, o); note_launch();
    if (ev) record_timing_event(ev[4], s);
}

}  // namespace

void launch_per_edge(const DevGraph &g, int64_t *out_dev, unsigned long long *pe_ws,
                     cudaStream_t s, cudaEvent_t *ev) {
    unsigned long long *peU = pe_ws, *peV = pe_ws + g.nE;
    if (g.nE > 0) cudaMemsetAsync(pe_ws, 0, (size_t)g.nE * 16, s);
    PvOut o{0, {peU, peV}};
    launch_pv_kernels(g, o, s, ev);
    if (g.nE == 0) return;
    const int64_t blocks = std::min<int64_t>((g.nE + edgerows::EDGES - 1) / edgerows::EDGES, 4096);
    k_pe_out<<<(unsigned)blocks, edgerows::THREADS, 0, s>>>(g, peU, peV, out_dev); note_launch();
}

void launch_per_vertex(const DevGraph &g, int64_t *out_dev, cudaStream_t s, cudaEvent_t *ev) {
    for (int sd = 0; sd < 2; sd++)
        if (g.side[sd].n > 0)
            cudaMemsetAsync(g.side[sd].pv, 0, (size_t)g.side[sd].n * 8, s);
    PvOut o{1, {nullptr, nullptr}};
    launch_pv_kernels(g, o, s, ev);
    for (int sd = 0; sd < 2; sd++) {
        const int64_t n = g.side[sd].n;
        if (n == 0) continue;
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
        k_pv_out<<<(unsigned)blocks, 256, 0, s>>>(g.side[sd], sd ? g.nU : 0, out_dev); note_launch();
    }
}

}  // namespace bb
