// count.cu - wedge aggregation and the C(.,2) reduction (Algorithm 2's
// counting loop and Lemma 2, made data parallel over anchors as in
// Algorithm 4; the anchor/endpoint roles are described in graph.cuh).
//
// For an anchor w every wedge w - v - u (v a neighbour of w, u in the suffix
// of v's row ranked above both) adds 1 to the symmetric tally of the pair
// (w, u) when sign(w,v) == sign(v,u) (Def. 5) and to the asymmetric tally
// otherwise (Def. 6). A pair with S symmetric and A asymmetric wedges holds
// C(S,2) + C(A,2) balanced and C(S+A,2) total butterflies (Lemma 2). Since
// C(n,2) = 0 + 1 + ... + (n-1), those sums are taken wedge by wedge: each
// wedge adds the count its own tally held before it (returned by the
// counter's atomic add) to the balanced sum and the count both tallies held
// to the total, which is exact in any order and needs no pass over the
// counters afterwards, only their reset.
//
// Work is spread by walkers: a team (a warp, or a whole CTA) loads a chunk
// of the anchor's middles, scans their suffix lengths and compacts the
// non-empty ones. The dense class's team_walk then steps through the
// chunk's wedges 32 at a time per warp (coalesced, one segment lookup per
// step); the other classes' lane_walk gives each thread an equal contiguous
// share of the chunk's wedges to stream through.
//
// Counters, per class (all in shared memory; S in bits 0..15, A in bits
// 16..31 of a u32, both bounded by the anchor's degree):
//   warp  - anchors of degree <= 255, one per warp: the hub window in
//           16-bit counters and an open-addressing hash (u64 slots:
//           endpoint + 1 in the high half) for the rest;
//   team  - medium anchors, one per 128-thread CTA: dense counters for the
//           hub window (top HUB_WINDOW ranks of the side, where most
//           endpoints fall) and a hash for the endpoints below the window;
//   ctah  - like team with a 512-thread CTA and an 8Ki-slot hash;
//   dense - heavy anchors with a short endpoint range: dense counters over
//           the whole range (walked in windows when longer than DENSE_CAP);
//           the heaviest are split over CTAs whose partial counts are
//           merged in global memory, adding the pairs formed across parts.
#include <algorithm>
#include <cstddef>
#include "graph.cuh"

namespace bb {

namespace {

constexpr int WARP_THREADS = 256;    // 8 independent warps per CTA
constexpr int TEAM_THREADS = 128;    // one team per CTA
constexpr int CTAH_THREADS = 512;
constexpr int DENSE_THREADS = 512;

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

// Per-thread partial sums are kept below 2^53 + 2^50 (larger ones go to the
// 128-bit accumulator at once; one anchor or job adds less than 2^50 to a
// thread's sums), so that the sum of up to 1024 threads' partials cannot
// wrap a u64 however large the graph's counts are.
__device__ __forceinline__ void spill_if_large(CountScratch *sc, unsigned long long &bal,
                                               unsigned long long &tot) {
    if ((bal | tot) >> 53) {
        acc_add(sc, bal, tot);
        bal = tot = 0;
    }
}

// adds the partial sums of a warp's threads to the accumulator
__device__ __forceinline__ void flush_warp(CountScratch *sc, unsigned long long bal,
                                           unsigned long long tot) {
    bal = warp_sum_u64(bal);
    tot = warp_sum_u64(tot);
    if (lane_id() == 0) acc_add(sc, bal, tot);
}

// contribution of one wedge given its pair's counts before it
__device__ __forceinline__ void wedge_terms(uint32_t oldS, uint32_t oldA, uint32_t asym,
                                            unsigned long long &bal, unsigned long long &tot) {
    bal += asym ? oldA : oldS;
    tot += oldS + oldA;
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

template <int TS>
__device__ __forceinline__ void team_sync() {
    if constexpr (TS == 32) __syncwarp();
    else __syncthreads();   // teams of more than one warp are whole CTAs
}

// A chunk of middles, compacted to those with a non-empty segment: the
// first entry of the segment in the other side's adjacency (absolute index,
// below 2^32 because nE is), and the wedges of the chunk before this middle
// (below 2^31) with the sign bit of the anchor's edge in bit 31.
struct Desc {
    uint32_t st;
    uint32_t excl_sw;
};

template <int TS>
struct alignas(16) WalkSmem {
    Desc desc[TS];
    uint32_t incl[TS];
    unsigned long long warp_part[TS / 32];  // per warp: wedges (low half), segments (high half)
    uint32_t tot[2];
    uint32_t item_next;               // next work item of the chunk (teams of several warps)
};

// wedges per work item when a team's warps share a chunk dynamically
constexpr uint32_t WALK_ITEM = 512;

// Walk the wedges of one anchor's middles [m0, m1) (its row starts at rb in
// the anchor side's descriptors smd; the middles' rows are in oadj) as a
// team of TS threads (t = thread index in the team). seg(md, st, len) picks
// the segment [st, st+len) of a middle's row from its descriptor;
// add(entry, sign bit of the anchor's edge to the middle) is called once per
// wedge (entry = endpoint side rank << 1 | sign of the middle-endpoint edge).
//
// Per chunk of TS middles the team scans the segment lengths and compacts
// the non-empty segments (their ends, incl[], are the chunk's wedge
// prefix); its warps then take WALK_ITEM-wedge slices of the chunk in turn (a
// lone warp takes the whole chunk). A warp walks its slice flat, 32
// consecutive wedges per step, lane l taking wedge base + l (coalesced
// loads). The step's wedges lie in at most 32 consecutive segments from
// `cur`, the segment of the step's first wedge: each lane reads one of
// their ends, the ends that fall inside the step form a bitmask, and a lane's
// segment is cur plus the ends at or before its wedge. When the whole step
// lies in segment cur (long segments) that reduces to one broadcast read.
template <int TS, int UNROLL = 4, typename Seg, typename Add>
__device__ __forceinline__ void team_walk(const uint4 *__restrict__ smd,
                                          const uint32_t *__restrict__ oadj, int64_t rb,
                                          uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                          Seg &&seg, Add &&add) {
    constexpr int NW = TS / 32;
    constexpr uint32_t EXMASK = 0x7fffffffu;
    const int lane = t & 31, w = t >> 5;
    const unsigned upto = (2u << lane) - 1u;   // bits 0..lane
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        const uint32_t j = mc + (uint32_t)t;
        long long st = 0;
        uint32_t len = 0, sw = 0;
        if (j < m1) {
            const uint4 d = smd[rb + j];
            sw = d.w;
            seg(d, st, len);
        }
        // inclusive team scan of the lengths; compacted index from a ballot
        uint32_t x = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, d);
            if (lane >= d) x += y;
        }
        const unsigned nzb = __ballot_sync(FULL, len > 0);
        uint32_t nzi = __popc(nzb & upto);
        if constexpr (NW > 1) {
            if (lane == 31) sm.warp_part[w] = x | ((unsigned long long)__popc(nzb) << 32);
            team_sync<TS>();
            uint32_t add_x = 0, add_n = 0;
            for (int k = 0; k < w; k++) {
                const unsigned long long v = sm.warp_part[k];
                add_x += (uint32_t)v;
                add_n += (uint32_t)(v >> 32);
            }
            x += add_x;
            nzi += add_n;
        }
        if (len > 0) {
            sm.desc[nzi - 1] = Desc{(uint32_t)st, (x - len) | (sw << 31)};
            sm.incl[nzi - 1] = x;
        }
        if (t == TS - 1) { sm.tot[0] = x; sm.tot[1] = nzi; sm.item_next = 0; }
        team_sync<TS>();
        const uint32_t T = sm.tot[0], NZ = sm.tot[1];
        // a warp takes the whole chunk when alone, else WALK_ITEM-wedge items in turn
        for (uint32_t item = 0;; item++) {
            uint32_t a, b;
            if constexpr (NW == 1) {
                if (item > 0) break;
                a = 0; b = T;
            } else {
                uint32_t it = 0;
                if (lane == 0) it = atomicAdd(&sm.item_next, 1u);
                it = __shfl_sync(FULL, it, 0);
                a = it * WALK_ITEM;
                if (a >= T) break;
                b = T - a > WALK_ITEM ? a + WALK_ITEM : T;
            }
            // segment holding wedge a: the first whose end is past a
            uint32_t cur = 0;
            if (a > 0) {
                uint32_t hi = NZ;
                while (cur < hi) {
                    const uint32_t mid = (cur + hi) >> 1;
                    if (sm.incl[mid] <= a) cur = mid + 1; else hi = mid;
                }
            }
            for (uint32_t base = a; base < b; base += 32u * UNROLL) {
                uint32_t addr[UNROLL], swq[UNROLL];
                bool ok[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; u++) {
                    const uint32_t bq = base + 32u * u;
                    ok[u] = false;
                    addr[u] = 0;
                    swq[u] = 0;
                    if (bq < b) {
                        const uint32_t ecur = sm.incl[cur];
                        uint32_t sg, nxt;
                        if (ecur >= bq + 32u) {  // the whole step is in segment cur
                            sg = cur;
                            nxt = ecur == bq + 32u ? cur + 1 : cur;
                        } else {
                            const uint32_t jj = cur + (uint32_t)lane;
                            const uint32_t p = (jj < NZ ? sm.incl[jj] : 0xffffffffu) - bq;  // >= 1
                            const unsigned M = __reduce_or_sync(FULL, p < 32u ? (1u << p) : 0u);
                            sg = cur + __popc(M & upto);
                            nxt = cur + __popc(__ballot_sync(FULL, p <= 32u));
                        }
                        const uint32_t q = bq + (uint32_t)lane;
                        if (q < b) {
                            const Desc dd = sm.desc[sg];
                            ok[u] = true;
                            addr[u] = dd.st + (q - (dd.excl_sw & EXMASK));
                            swq[u] = dd.excl_sw >> 31;
                        }
                        cur = nxt;
                    }
                }
                uint32_t xv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; u++)
                    if (ok[u]) xv[u] = oadj[addr[u]];
#pragma unroll
                for (int u = 0; u < UNROLL; u++)
                    if (ok[u]) add(xv[u], swq[u]);
            }
        }
        team_sync<TS>();
    }
}

// Lane walker. After the same chunk scan and compaction, each thread takes
// an equal contiguous part [a, b) of the chunk's flat wedge range and
// streams through it, stepping to the next segment when one ends: no
// per-step segment search, and the threads of a team get equal wedge
// counts. Used where anchors are small or medium (warp, team and CTA-hash
// classes); the dense class keeps team_walk's coalesced steps.
template <int U, typename Add>
__device__ __forceinline__ void lane_range(const uint32_t *__restrict__ oadj, const Desc *desc,
                                           const uint32_t *incl, uint32_t NZ, uint32_t a,
                                           uint32_t b, Add &&add) {
    constexpr uint32_t EXMASK = 0x7fffffffu;
    if (a >= b) return;
    uint32_t k = 0, hi = NZ;  // segment holding wedge a
    while (k < hi) {
        const uint32_t mid = (k + hi) >> 1;
        if (incl[mid] <= a) k = mid + 1; else hi = mid;
    }
    Desc d = desc[k];
    uint32_t ex = d.excl_sw & EXMASK;
    uint32_t p = d.st + (a - ex);
    uint32_t pend = d.st + (incl[k] - ex);
    uint32_t cs = d.excl_sw >> 31;
    auto next_segment = [&]() {
        k++;
        d = desc[k];
        ex = d.excl_sw & EXMASK;
        p = d.st;
        pend = d.st + (incl[k] - ex);
        cs = d.excl_sw >> 31;
    };
    uint32_t i = a;
    for (; i + U <= b; i += U) {
        uint32_t pa[U], sq[U];
        if (pend - p >= U) {  // the U wedges lie in the current segment
#pragma unroll
            for (int u = 0; u < U; u++) { pa[u] = p + u; sq[u] = cs; }
            p += U;
        } else {
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (p == pend) next_segment();
                pa[u] = p++;
                sq[u] = cs;
            }
        }
        uint32_t xv[U];
#pragma unroll
        for (int u = 0; u < U; u++) xv[u] = oadj[pa[u]];
#pragma unroll
        for (int u = 0; u < U; u++) add(xv[u], sq[u]);
    }
    for (; i < b; i++) {
        if (p == pend) next_segment();
        const uint32_t x = oadj[p++];
        add(x, cs);
    }
}

// equal share t of n among TS threads
template <int TS>
__device__ __forceinline__ uint32_t share(uint32_t n, uint32_t t) {
    return (uint32_t)((unsigned long long)n * t / TS);
}

template <int TS, int U = 4, typename Seg, typename Add>
__device__ __forceinline__ void lane_walk(const uint4 *__restrict__ smd,
                                          const uint32_t *__restrict__ oadj, int64_t rb,
                                          uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                          Seg &&seg, Add &&add) {
    constexpr int NW = TS / 32;
    const int lane = t & 31, w = t >> 5;
    const unsigned upto = (2u << lane) - 1u;
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        const uint32_t j = mc + (uint32_t)t;
        long long st = 0;
        uint32_t len = 0, sw = 0;
        if (j < m1) {
            const uint4 d = smd[rb + j];
            sw = d.w;
            seg(d, st, len);
        }
        uint32_t x = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, d);
            if (lane >= d) x += y;
        }
        const unsigned nzb = __ballot_sync(FULL, len > 0);
        uint32_t nzi = __popc(nzb & upto);
        if constexpr (NW > 1) {
            if (lane == 31) sm.warp_part[w] = x | ((unsigned long long)__popc(nzb) << 32);
            team_sync<TS>();
            uint32_t add_x = 0, add_n = 0;
            for (int k = 0; k < w; k++) {
                const unsigned long long v = sm.warp_part[k];
                add_x += (uint32_t)v;
                add_n += (uint32_t)(v >> 32);
            }
            x += add_x;
            nzi += add_n;
        }
        if (len > 0) {
            sm.desc[nzi - 1] = Desc{(uint32_t)st, (x - len) | (sw << 31)};
            sm.incl[nzi - 1] = x;
        }
        if (t == TS - 1) { sm.tot[0] = x; sm.tot[1] = nzi; }
        team_sync<TS>();
        const uint32_t T = sm.tot[0], NZ = sm.tot[1];
        lane_range<U>(oadj, sm.desc, sm.incl, NZ, share<TS>(T, t), share<TS>(T, t + 1), add);
        team_sync<TS>();
    }
}

// One warp, two segment families of the same middles (the hub-window part
// and the part below it) from one chunk scan: each lane walks its share of
// the first family with addA, then its share of the second with addB.
template <int U = 4, typename SegA, typename AddA, typename SegB, typename AddB>
__device__ __forceinline__ void lane_walk2(const uint4 *__restrict__ smd,
                                           const uint32_t *__restrict__ oadj, int64_t rb,
                                           uint32_t m0, uint32_t m1, WalkSmem<32> &sa,
                                           WalkSmem<32> &sb, int lane, SegA &&sega, AddA &&adda,
                                           SegB &&segb, AddB &&addb) {
    const unsigned upto = (2u << lane) - 1u;
    for (uint32_t mc = m0; mc < m1; mc += 32) {
        const uint32_t j = mc + (uint32_t)lane;
        long long sta = 0, stb = 0;
        uint32_t la = 0, lb = 0, sw = 0;
        if (j < m1) {
            const uint4 d = smd[rb + j];
            sw = d.w;
            sega(d, sta, la);
            segb(d, stb, lb);
        }
        unsigned long long x = (unsigned long long)la | ((unsigned long long)lb << 32);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, x, d);
            if (lane >= d) x += y;
        }
        const uint32_t xa = (uint32_t)x, xb = (uint32_t)(x >> 32);
        const unsigned nza = __ballot_sync(FULL, la > 0), nzb = __ballot_sync(FULL, lb > 0);
        if (la > 0) {
            const uint32_t i = __popc(nza & upto) - 1;
            sa.desc[i] = Desc{(uint32_t)sta, (xa - la) | (sw << 31)};
            sa.incl[i] = xa;
        }
        if (lb > 0) {
            const uint32_t i = __popc(nzb & upto) - 1;
            sb.desc[i] = Desc{(uint32_t)stb, (xb - lb) | (sw << 31)};
            sb.incl[i] = xb;
        }
        const uint32_t TA = __shfl_sync(FULL, xa, 31), TB = __shfl_sync(FULL, xb, 31);
        __syncwarp();
        lane_range<U>(oadj, sa.desc, sa.incl, __popc(nza), share<32>(TA, lane),
                      share<32>(TA, lane + 1), adda);
        lane_range<U>(oadj, sb.desc, sb.incl, __popc(nzb), share<32>(TB, lane),
                      share<32>(TB, lane + 1), addb);
        __syncwarp();
    }
}

// insert-or-increment in a shared-memory table of 2^(32-shift) u64 slots;
// returns the packed (S | A << 16) count the key held before
__device__ __forceinline__ uint32_t hash_add(unsigned long long *tab, uint32_t shift,
                                             uint32_t mask, uint32_t key, uint32_t inc,
                                             uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        unsigned long long cur = *((volatile unsigned long long *)&tab[h]);
        uint32_t k = (uint32_t)(cur >> 32);
        if (k == key) return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
        if (k == 0) {
            unsigned long long want = ((unsigned long long)key << 32) | inc;
            unsigned long long old = atomicCAS(&tab[h], 0ull, want);
            if (old == 0ull) return 0u;
            if ((uint32_t)(old >> 32) == key)
                return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
        }
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
    return 0u;
}

// hash add plus the wedge's contribution
__device__ __forceinline__ void hash_wedge(unsigned long long *tab, uint32_t shift, uint32_t mask,
                                           uint32_t u, uint32_t asym, uint32_t *err,
                                           unsigned long long &bal, unsigned long long &tot) {
    const uint32_t old = hash_add(tab, shift, mask, u + 1, asym ? INC_ASYM : INC_SYM, err);
    wedge_terms(old & 0xffffu, old >> 16, asym, bal, tot);
}

// the same with 32-bit running sums (anchors whose sums provably fit):
// dp2a takes the previous S or A (16-bit halves of the slot's count) or both
__device__ __forceinline__ void hash_wedge32(unsigned long long *tab, uint32_t shift,
                                             uint32_t mask, uint32_t x, uint32_t sw,
                                             uint32_t *err, uint32_t &b32, uint32_t &t32) {
    const uint32_t asym = (x ^ sw) & 1u;
    const uint32_t old = hash_add(tab, shift, mask, (x >> 1) + 1, asym ? INC_ASYM : INC_SYM, err);
    b32 = __dp2a_lo(old, 1u << (asym << 3), b32);
    t32 = __dp2a_lo(old, 0x0101u, t32);
}

// zero the first `cap` slots of a table (cap a multiple of 2) as a team
template <int TS>
__device__ __forceinline__ void clear_table(unsigned long long *tab, uint32_t cap, int t) {
    ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tab);
    for (uint32_t i = t; i < cap / 2; i += TS) t2[i] = make_ulonglong2(0ull, 0ull);
}

// table of 2^k slots, 2^k >= max(min_cap, 2 need + 1), at most max_cap (load <= 1/2
// unless capped: linear probes stay short)
__device__ __forceinline__ void table_geometry(uint64_t need, uint32_t min_cap, uint32_t max_cap,
                                               uint32_t &cap, uint32_t &shift) {
    uint64_t want = 2 * need + 1;
    cap = min_cap;
    shift = 32 - (31 - __clz(min_cap));
    while ((uint64_t)cap < want && cap < max_cap) { cap <<= 1; shift--; }
}

// The few values one anchor's walk needs (anchor side S, middle side O).
struct Anchor {
    const uint4 *smd;
    const uint32_t *oadj;
    int64_t rb, ns;
    uint32_t r, deg;
    uint64_t W, wnh;
};

__device__ __forceinline__ Anchor load_anchor(const DevGraph &G, const AnchorRec &rec) {
    Anchor a;
    const bool v = rec.anchor & 1u;
    a.smd = v ? G.side[1].md : G.side[0].md;
    a.oadj = v ? G.side[0].adj : G.side[1].adj;
    a.ns = v ? G.side[1].n : G.side[0].n;
    a.r = rec.anchor >> 1;
    a.rb = rec.rb;
    a.deg = rec.deg;
    a.W = rec.W;
    a.wnh = rec.wnh;
    return a;
}

// the whole wedge suffix of a middle
struct FullSeg {
    __device__ void operator()(const uint4 &d, long long &st, uint32_t &len) const {
        st = d.x;
        len = d.z - d.x;
    }
};

// the part of a middle's suffix inside the hub window
struct HubSeg {
    __device__ void operator()(const uint4 &d, long long &st, uint32_t &len) const {
        st = d.y;
        len = d.z - d.y;
    }
};

// the part of a middle's suffix below the hub window
struct LowSeg {
    __device__ void operator()(const uint4 &d, long long &st, uint32_t &len) const {
        st = d.x;
        len = d.y - d.x;
    }
};

// ------------------------------------------------------------ warp class
// Per warp: the hub window as 16-bit counters, two per word (S in the low
// byte, A in the high byte; both <= the anchor's degree <= 255), a small
// hash for endpoints below the window, and the walker's chunk.
struct alignas(16) WarpSmem {
    uint32_t win[HUB_WINDOW / 2];
    unsigned long long tab[WARP_CAP];
    WalkSmem<32> walk, walk2;  // hub-window and below-window segments
};

// per-warp copies are laid out back to back and reset with 16-byte stores
static_assert(sizeof(WarpSmem) % 16 == 0, "WarpSmem must keep 16-byte alignment");
static_assert((HUB_WINDOW & (HUB_WINDOW - 1)) == 0, "hub window indexes are masked");
static_assert(offsetof(WarpSmem, tab) % 16 == 0, "table needs 16-byte alignment");

// anchors with at least this many wedges walk eight wedges per lane step
// (more loads in flight) in the single-graph kernel
constexpr uint64_t WARP_WIDE_W = 2048;

// one warp-class anchor, walked by one warp; WIDE: large anchors take the
// eight-wedge lane steps (the batch kernel, whose mix is mostly small
// anchors, keeps four: the second walker instance slows it)
template <bool WIDE>
__device__ __forceinline__ void warp_anchor(const DevGraph &G, WarpSmem &sm, const AnchorRec &rec,
                                            unsigned lane, unsigned long long &bal,
                                            unsigned long long &tot) {
    uint32_t *err = &G.scratch->err;
    const Anchor A = load_anchor(G, rec);
    const uint64_t W = A.W, above = (uint64_t)(A.ns - A.r - 1);
    uint32_t cap = 0, shift = 0;
    // 32-bit sums: a lane walks at most W/32 + 1 <= 513 wedges of each
    // family of the anchor, each adding at most 2 * 255
    uint32_t b32 = 0, t32 = 0;
    if (W <= WARP_SMALL_W) {  // hash every endpoint
        table_geometry(W < above ? W : above, 32, WARP_CAP, cap, shift);
        const uint32_t mask = cap - 1;
        lane_walk<32>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, (int)lane, FullSeg{},
                      [&](uint32_t x, uint32_t sw) {
                          hash_wedge32(sm.tab, shift, mask, x, sw, err, b32, t32);
                      });
    } else {
        const int64_t ns = A.ns;
        const uint32_t wb = ns > (int64_t)HUB_WINDOW ? (uint32_t)(ns - HUB_WINDOW) : 0u;
        const uint32_t wb2 = wb << 1;  // the window base as an entry (side ranks < 2^31)
        const uint64_t wnh = A.wnh;
        const uint64_t above_nh = wb > A.r + 1 ? (uint64_t)wb - A.r - 1 : 0;
        if (wnh > 0) table_geometry(wnh < above_nh ? wnh : above_nh, 32, WARP_CAP, cap, shift);
        const uint32_t mask = cap - 1;
        uint32_t bad_off = 0;
        auto hub_add = [&](uint32_t x, uint32_t sw) {
            // S in byte 0 and A in byte 1 of the endpoint's 16-bit half of a
            // word (both <= the degree <= 255). The entry less twice the
            // window base is 2 * (window index) + sign: bit 1 picks the half
            // and bit 0 xor the anchor edge's sign the byte. The increment is
            // that byte's lowest bit; as a byte mask for dp4a it picks the
            // tally's own previous value out of the returned word, and
            // 0x0101 at the half picks S + A.
            const uint32_t xi = x - wb2;
            bad_off |= xi;  // any entry outside the window sets a high bit
            const uint32_t sh = ((xi ^ sw) & 3u) << 3;
            const uint32_t inc = 1u << sh;
            const uint32_t old = atomicAdd(&sm.win[(xi >> 2) & (HUB_WINDOW / 2 - 1)], inc);
            b32 = __dp4a(old, inc, b32);
            t32 = __dp4a(old, 0x0101u << (sh & 16u), t32);
        };
        auto low_add = [&](uint32_t x, uint32_t sw) {
            hash_wedge32(sm.tab, shift, mask, x, sw, err, b32, t32);
        };
        if (WIDE && W >= WARP_WIDE_W)
            lane_walk2<8>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, (int)lane, HubSeg{},
                          hub_add, LowSeg{}, low_add);
        else
            lane_walk2<4>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, (int)lane, HubSeg{},
                          hub_add, LowSeg{}, low_add);
        if (bad_off >= 2 * HUB_WINDOW) set_error(err, E_INTERNAL);
        // reset the window words an endpoint can have reached
        const uint32_t first = (A.r + 1 > wb ? A.r + 1 - wb : 0u) >> 3;  // uint4 index
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = first + lane; q < HUB_WINDOW / 8; q += 32)
            w4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    bal += b32;
    tot += t32;
    clear_table<32>(sm.tab, cap, (int)lane);
    __syncwarp();
}

__device__ __forceinline__ WarpSmem &warp_smem_init(unsigned char *smem_raw, unsigned lane) {
    WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[threadIdx.x >> 5];
    clear_table<32>(sm.tab, WARP_CAP, (int)lane);
    for (uint32_t i = lane; i < HUB_WINDOW / 2; i += 32) sm.win[i] = 0u;
    __syncwarp();
    return sm;
}

__global__ void __launch_bounds__(WARP_THREADS, 3) k_warp(DevGraph G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned lane = lane_id();
    WarpSmem &sm = warp_smem_init(smem_raw, lane);
    const uint32_t n = G.ctr[CTR_WARP];
    const uint32_t gw = (blockIdx.x * WARP_THREADS + threadIdx.x) >> 5;
    const uint32_t GW = (gridDim.x * WARP_THREADS) >> 5;
    unsigned long long bal = 0, tot = 0;
    for (uint32_t idx = gw; idx < n; idx += GW) {
        warp_anchor<true>(G, sm, G.warp_list[idx], lane, bal, tot);
        spill_if_large(G.scratch, bal, tot);
    }
    flush_warp(G.scratch, bal, tot);
}

// ------------------------------------------------- team and CTA-hash classes
template <int TS, uint32_t HCAP>
struct alignas(16) HybSmem {
    uint32_t win[HUB_WINDOW];          // hub window counters
    unsigned long long tab[HCAP];      // hash for endpoints below the window
    WalkSmem<TS> walk;
    uint32_t job;
};

template <int TS, uint32_t HCAP>
__device__ __forceinline__ HybSmem<TS, HCAP> &hybrid_smem_init(unsigned char *smem_raw) {
    using Smem = HybSmem<TS, HCAP>;
    static_assert(offsetof(Smem, tab) % 16 == 0, "table needs 16-byte alignment");
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    for (uint32_t i = threadIdx.x; i < HUB_WINDOW; i += TS) sm.win[i] = 0;
    clear_table<TS>(sm.tab, HCAP, (int)threadIdx.x);
    return sm;
}

// one team/CTA-hash anchor, walked by the whole CTA
template <int TS, uint32_t HCAP>
__device__ __forceinline__ void hybrid_anchor(const DevGraph &G, HybSmem<TS, HCAP> &sm,
                                              const AnchorRec &rec, unsigned long long &bal,
                                              unsigned long long &tot) {
    const int t = threadIdx.x;
    uint32_t *err = &G.scratch->err;
    const Anchor A = load_anchor(G, rec);
    const int64_t ns = A.ns;
    const uint32_t wb = ns > (int64_t)HUB_WINDOW ? (uint32_t)(ns - HUB_WINDOW) : 0u;
    const uint64_t W = A.W, wnh = A.wnh;
    const uint64_t above_nh = wb > A.r + 1 ? (uint64_t)wb - A.r - 1 : 0;
    // lane steps: four wedges for team anchors (more register pressure
    // costs them occupancy), eight for the CTA-hash class
    constexpr int LU = TS == TEAM_THREADS ? 4 : 8;
    if (W > wnh) {  // endpoints inside the hub window
        // Team anchors (at most TEAM_W_MAX wedges, each adding at most
        // 2 * 65535) sum the hub part in 32 bits: dp2a takes the previous
        // S or A (16-bit halves of the returned word) or their sum.
        constexpr bool narrow = TS == TEAM_THREADS;
        static_assert(!narrow || TEAM_W_MAX * 2 * 65535 < (1ull << 32), "32-bit team sums");
        uint32_t b32 = 0, t32 = 0;
        lane_walk<TS, LU>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, HubSeg{},
                      [&](uint32_t x, uint32_t sw) {
                          const uint32_t asym = (x ^ sw) & 1u;
                          const uint32_t idx = (x >> 1) - wb;
                          if (idx >= HUB_WINDOW) { set_error(err, E_INTERNAL); return; }
                          const uint32_t old = atomicAdd(&sm.win[idx], asym ? INC_ASYM : INC_SYM);
                          if constexpr (narrow) {
                              b32 = __dp2a_lo(old, 1u << (asym << 3), b32);
                              t32 = __dp2a_lo(old, 0x0101u, t32);
                          } else {
                              wedge_terms(old & 0xffffu, old >> 16, asym, bal, tot);
                          }
                      });
        bal += b32;
        tot += t32;
    }
    uint32_t cap = 0;
    if (wnh > 0) {  // endpoints below the window
        uint32_t shift;
        table_geometry(wnh < above_nh ? wnh : above_nh, 32, HCAP, cap, shift);
        const uint32_t mask = cap - 1;
        lane_walk<TS, LU>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, LowSeg{},
                      [&](uint32_t x, uint32_t sw) {
                          hash_wedge(sm.tab, shift, mask, x >> 1, (x ^ sw) & 1u, err, bal, tot);
                      });
    }
    __syncthreads();
    if (W > wnh) {
        const uint32_t first = (A.r + 1 > wb ? A.r + 1 - wb : 0u) >> 2;  // uint4 index
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = first + t; q < HUB_WINDOW / 4; q += TS)
            w4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    clear_table<TS>(sm.tab, cap, t);
}

template <int TS, uint32_t HCAP, int CTR, int CLS>
__device__ __forceinline__ void hybrid_body(DevGraph &G, const AnchorRec *list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HybSmem<TS, HCAP> &sm = hybrid_smem_init<TS, HCAP>(smem_raw);
    const uint32_t n = G.ctr[CTR];
    unsigned long long bal = 0, tot = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(&G.scratch->job_next[CLS], 1u);
        __syncthreads();
        const uint32_t jid = sm.job;
        __syncthreads();
        if (jid >= n) break;
        hybrid_anchor<TS, HCAP>(G, sm, list[jid], bal, tot);
        spill_if_large(G.scratch, bal, tot);
    }
    block_sum2<TS>(bal, tot);
    if (threadIdx.x == 0) acc_add(G.scratch, bal, tot);
}

__global__ void __launch_bounds__(TEAM_THREADS) k_team(DevGraph G) {
    hybrid_body<TEAM_THREADS, TEAM_CAP, CTR_TEAM, CLS_TEAM>(G, G.team_list);
}

__global__ void __launch_bounds__(CTAH_THREADS) k_ctah(DevGraph G) {
    hybrid_body<CTAH_THREADS, CTAH_CAP, CTR_CTAH, CLS_CTAH>(G, G.ctah_list);
}

// ------------------------------------------------------------ dense class
struct alignas(16) DenseSmem {
    uint32_t cnt[DENSE_CAP];
    WalkSmem<DENSE_THREADS> walk;
    uint32_t job, last;
};

// one dense job (an anchor, or one middle slice of a split anchor), walked
// by the whole CTA; adds each thread's part of its sums to bal and tot
__device__ __forceinline__ void dense_job(const DevGraph &G, DenseSmem &sm, const DenseJob &J,
                                          unsigned long long &bal, unsigned long long &tot) {
    const int t = threadIdx.x;
    CountScratch *sc = G.scratch;
    const bool sv = J.anchor & 1u;
    const SideCSR &S = sv ? G.side[1] : G.side[0];
    AnchorRec rec;
    rec.anchor = J.anchor;
    rec.rb = (uint32_t)S.off[J.anchor >> 1];
    rec.deg = 0; rec.W = 0; rec.wnh = 0;
    const Anchor A = load_anchor(G, rec);
    const uint32_t e_lo = A.r + 1, e_hi = (uint32_t)A.ns;
    const bool windows = (e_hi - e_lo) > DENSE_CAP;
    for (uint32_t e0 = e_lo; e0 < e_hi; e0 += DENSE_CAP) {
        const uint32_t e1 = e_hi - e0 > DENSE_CAP ? e0 + DENSE_CAP : e_hi;
        const uint32_t len = e1 - e0;
        for (uint32_t i = t; i < len; i += DENSE_THREADS) sm.cnt[i] = 0;
        __syncthreads();
        auto add = [&](uint32_t x, uint32_t sw) {
            const uint32_t asym = (x ^ sw) & 1u;
            const uint32_t idx = (x >> 1) - e0;
            if (idx >= len) { set_error(&sc->err, E_INTERNAL); return; }
            const uint32_t old = atomicAdd(&sm.cnt[idx], asym ? INC_ASYM : INC_SYM);
            wedge_terms(old & 0xffffu, old >> 16, asym, bal, tot);
        };
        if (windows) {
            team_walk<DENSE_THREADS>(
                A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t,
                [&](const uint4 &d, long long &st, uint32_t &l) {
                    const long long s0 = lower_bound_u32(A.oadj, d.x, d.z, e0 << 1);
                    st = s0;
                    l = (uint32_t)(lower_bound_u32(A.oadj, s0, d.z, e1 << 1) - s0);
                },
                add);
        } else {
            team_walk<DENSE_THREADS>(A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t, FullSeg{}, add);
        }
        if (J.group != NO_GROUP) {
            // merge this part's counts into the group's global counters; a
            // count p added to c already there closes c*p new pairs
            const SplitGroup grp = G.groups[J.group];
            uint32_t *part = G.gpart + grp.goff;
            __syncthreads();
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
            // the last part to arrive resets the group's counters
            __threadfence();
            __syncthreads();
            if (t == 0) {
                const uint32_t ticket = atomicAdd(&G.gdone[J.group], 1u);
                sm.last = ticket == grp.parts - 1 ? 1u : 0u;
            }
            __syncthreads();
            if (sm.last) {
                __threadfence();
                for (uint32_t i = t; i < len; i += DENSE_THREADS) part[i] = 0;
                if (t == 0) G.gdone[J.group] = 0;
            }
        }
        __syncthreads();  // the next window or job rewrites the counters
    }
}

__global__ void __launch_bounds__(DENSE_THREADS) k_dense(DevGraph G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DenseSmem &sm = *reinterpret_cast<DenseSmem *>(smem_raw);
    const uint32_t njobs = G.ctr[CTR_DENSE];
    unsigned long long bal = 0, tot = 0;  // summed over all jobs of this CTA
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(&G.scratch->job_next[CLS_DENSE], 1u);
        __syncthreads();
        const uint32_t jid = sm.job;
        __syncthreads();
        if (jid >= njobs) break;
        dense_job(G, sm, G.dense_jobs[jid], bal, tot);
        spill_if_large(G.scratch, bal, tot);
    }
    flush_warp(G.scratch, bal, tot);
}

// ---------------------------------------------------- batched (many graphs)
// The same per-item work over the items of many resident graphs at once:
// items of class c of graph i are numbered prefix[c][i] .. prefix[c][i+1)-1
// in one space and handed out from a cursor per class. Sums go to each
// item's own graph.
struct BatchArgs {
    const DevGraph *graphs;
    const uint32_t *prefix;   // [NCLS][n + 1]
    uint32_t *next;           // [NCLS] item cursors, zeroed before the launch
    uint32_t n;
    uint32_t warp_chunk;      // anchors a warp takes per grab
};

__device__ __forceinline__ uint32_t batch_graph_of(const uint32_t *p, uint32_t n, uint32_t item) {
    uint32_t lo = 0, hi = n;  // last i with p[i] <= item (p[0] = 0 <= item < p[n])
    while (hi - lo > 1) {
        const uint32_t m = (lo + hi) >> 1;
        if (p[m] <= item) lo = m; else hi = m;
    }
    return lo;
}

__global__ void __launch_bounds__(WARP_THREADS, 4) k_warp_batch(BatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned lane = lane_id();
    WarpSmem &sm = warp_smem_init(smem_raw, lane);
    const uint32_t *p = B.prefix + (size_t)CLS_WARP * (B.n + 1);
    const uint32_t total = p[B.n];
    for (;;) {
        uint32_t c0 = 0;
        if (lane == 0) c0 = atomicAdd(&B.next[CLS_WARP], B.warp_chunk);
        c0 = __shfl_sync(FULL, c0, 0);
        if (c0 >= total) break;
        const uint32_t c1 = total - c0 > B.warp_chunk ? c0 + B.warp_chunk : total;
        uint32_t gi = batch_graph_of(p, B.n, c0);
        uint32_t gbeg = p[gi], gend = p[gi + 1];
        unsigned long long bal = 0, tot = 0;
        for (uint32_t it = c0; it < c1; it++) {
            if (it >= gend) {  // next graph (skipping any without items): flush this one
                bal = warp_sum_u64(bal); tot = warp_sum_u64(tot);
                if (lane == 0) acc_add(B.graphs[gi].scratch, bal, tot);
                bal = tot = 0;
                do { gi++; gbeg = gend; gend = p[gi + 1]; } while (it >= gend);
            }
            const DevGraph &G = B.graphs[gi];
            warp_anchor<false>(G, sm, G.warp_list[it - gbeg], lane, bal, tot);
        }
        bal = warp_sum_u64(bal); tot = warp_sum_u64(tot);
        if (lane == 0) acc_add(B.graphs[gi].scratch, bal, tot);
    }
}

template <int TS, uint32_t HCAP, int CLS>
__device__ __forceinline__ void hybrid_batch_body(const BatchArgs &B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HybSmem<TS, HCAP> &sm = hybrid_smem_init<TS, HCAP>(smem_raw);
    const uint32_t *p = B.prefix + (size_t)CLS * (B.n + 1);
    const uint32_t total = p[B.n];
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(&B.next[CLS], 1u);
        __syncthreads();
        const uint32_t it = sm.job;
        __syncthreads();
        if (it >= total) break;
        const uint32_t gi = batch_graph_of(p, B.n, it);
        const DevGraph &G = B.graphs[gi];
        const AnchorRec *list = CLS == CLS_TEAM ? G.team_list : G.ctah_list;
        unsigned long long bal = 0, tot = 0;
        hybrid_anchor<TS, HCAP>(G, sm, list[it - p[gi]], bal, tot);
        block_sum2<TS>(bal, tot);
        if (threadIdx.x == 0) acc_add(G.scratch, bal, tot);
    }
}

__global__ void __launch_bounds__(TEAM_THREADS) k_team_batch(BatchArgs B) {
    hybrid_batch_body<TEAM_THREADS, TEAM_CAP, CLS_TEAM>(B);
}

__global__ void __launch_bounds__(CTAH_THREADS) k_ctah_batch(BatchArgs B) {
    hybrid_batch_body<CTAH_THREADS, CTAH_CAP, CLS_CTAH>(B);
}

__global__ void __launch_bounds__(DENSE_THREADS) k_dense_batch(BatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DenseSmem &sm = *reinterpret_cast<DenseSmem *>(smem_raw);
    const uint32_t *p = B.prefix + (size_t)CLS_DENSE * (B.n + 1);
    const uint32_t total = p[B.n];
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(&B.next[CLS_DENSE], 1u);
        __syncthreads();
        const uint32_t it = sm.job;
        __syncthreads();
        if (it >= total) break;
        const uint32_t gi = batch_graph_of(p, B.n, it);
        const DevGraph &G = B.graphs[gi];
        unsigned long long bal = 0, tot = 0;
        dense_job(G, sm, G.dense_jobs[it - p[gi]], bal, tot);
        block_sum2<DENSE_THREADS>(bal, tot);
        if (threadIdx.x == 0) acc_add(G.scratch, bal, tot);
    }
}

// zero every graph's count scratch and the class cursors
__global__ void k_batch_prep(BatchArgs B) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NCLS) B.next[i] = 0;
    for (uint32_t g = i; g < B.n; g += gridDim.x * blockDim.x) {
        CountScratch *sc = B.graphs[g].scratch;
        for (int k = 0; k < 4; k++) sc->acc[k] = 0;
        for (int k = 0; k < 5; k++) sc->job_next[k] = 0;
        sc->err = 0;
    }
}

// per graph, BATCH_OUT words: balanced lo/hi, total lo/hi, count error |
// build error << 32
__global__ void k_batch_results(BatchArgs B, unsigned long long *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n; i += gridDim.x * blockDim.x) {
        const DevGraph &G = B.graphs[i];
        unsigned long long *o = out + (size_t)i * BATCH_OUT;
        for (int k = 0; k < 4; k++) o[k] = G.scratch->acc[k];
        o[4] = (unsigned long long)G.scratch->err | ((unsigned long long)*G.err << 32);
    }
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
        const SideCSR &U = G.side[0];
        const SideCSR &V = G.side[1];
        uint32_t ru = U.sr_of_id[lo];
        uint32_t rv = V.sr_of_id[G.col[e]];
        int64_t p = lower_bound_u32(U.adj, U.off[ru], U.off[ru + 1], rv << 1);
        int64_t q = lower_bound_u32(V.adj, V.off[rv], V.off[rv + 1], ru << 1);
        atomicXor(&U.adj[p], 1u);
        atomicXor(&V.adj[q], 1u);
        atomicXor(&U.md[p].w, 1u);   // the descriptors carry the edge's sign too
        atomicXor(&V.md[q].w, 1u);
    }
}

constexpr size_t WARP_SMEM = (WARP_THREADS / 32) * sizeof(WarpSmem);
constexpr size_t TEAM_SMEM = sizeof(HybSmem<TEAM_THREADS, TEAM_CAP>);
constexpr size_t CTAH_SMEM = sizeof(HybSmem<CTAH_THREADS, CTAH_CAP>);
constexpr size_t DENSE_SMEM = sizeof(DenseSmem);


struct LaunchCfg {
    int warp_blocks = 0, team_blocks = 0, ctah_blocks = 0, dense_blocks = 0;
    int batch_blocks[NCLS] = {};
    int sms = 0;
};

LaunchCfg g_cfg;
int g_cfg_device = -1;

template <typename K>
int blocks_for(K kernel, int threads, size_t smem, int sms) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem);
    return std::max(1, b) * sms;
}

void init_cfg() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_cfg_device == dev) return;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    const int sms = prop.multiProcessorCount;
    g_cfg.sms = sms;
    g_cfg.warp_blocks = blocks_for(k_warp, WARP_THREADS, WARP_SMEM, sms);
    g_cfg.team_blocks = blocks_for(k_team, TEAM_THREADS, TEAM_SMEM, sms);
    g_cfg.ctah_blocks = blocks_for(k_ctah, CTAH_THREADS, CTAH_SMEM, sms);
    g_cfg.dense_blocks = blocks_for(k_dense, DENSE_THREADS, DENSE_SMEM, sms);
    g_cfg.batch_blocks[CLS_WARP] = blocks_for(k_warp_batch, WARP_THREADS, WARP_SMEM, sms);
    g_cfg.batch_blocks[CLS_TEAM] = blocks_for(k_team_batch, TEAM_THREADS, TEAM_SMEM, sms);
    g_cfg.batch_blocks[CLS_CTAH] = blocks_for(k_ctah_batch, CTAH_THREADS, CTAH_SMEM, sms);
    g_cfg.batch_blocks[CLS_DENSE] = blocks_for(k_dense_batch, DENSE_THREADS, DENSE_SMEM, sms);
    g_cfg_device = dev;
}

}  // namespace

void count_init() { init_cfg(); }

void launch_count(const DevGraph &g, cudaStream_t s, int64_t *per_vertex_dev, cudaEvent_t *ev) {
    (void)per_vertex_dev;
    init_cfg();
    cudaMemsetAsync(g.scratch, 0, sizeof(CountScratch), s);
    if (ev) record_timing_event(ev[0], s);
    k_dense<<<g_cfg.dense_blocks, DENSE_THREADS, DENSE_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[1], s);
    k_ctah<<<g_cfg.ctah_blocks, CTAH_THREADS, CTAH_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[2], s);
    k_team<<<g_cfg.team_blocks, TEAM_THREADS, TEAM_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[3], s);
    k_warp<<<g_cfg.warp_blocks, WARP_THREADS, WARP_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[4], s);
}

int batch_max_blocks(int cls) {
    init_cfg();
    return g_cfg.batch_blocks[cls];
}

void launch_count_batch(const BatchLaunch &L, const BatchTune &T, cudaStream_t s,
                        const cudaStream_t *side, const cudaEvent_t *ev, const cudaEvent_t *tev) {
    init_cfg();
    BatchArgs B;
    B.graphs = L.graphs;
    B.prefix = L.prefix;
    B.next = L.next;
    B.n = L.n;
    B.warp_chunk = T.warp_chunk ? T.warp_chunk : 1;
    const uint32_t prep_blocks = std::min<uint32_t>((L.n + 255) / 256 + 1, 1024);
    k_batch_prep<<<prep_blocks, 256, 0, s>>>(B); note_launch();
    // classes in descending item size, so the long dense jobs start first
    const int order[NCLS] = {CLS_DENSE, CLS_CTAH, CLS_TEAM, CLS_WARP};
    int nlaunch = 0;
    for (int k = 0; k < NCLS; k++) nlaunch += L.items[order[k]] ? 1 : 0;
    const bool conc = T.concurrent && side && ev && nlaunch > 1 && !tev;
    if (conc) {  // fork exactly the side streams that get a kernel (a capture must join them all)
        cudaEventRecord(ev[0], s);
        for (int k = 0; k + 1 < nlaunch; k++) cudaStreamWaitEvent(side[k], ev[0], 0);
    }
    int used = 0;
    for (int k = 0; k < NCLS; k++) {
        const int c = order[k];
        if (tev) cudaEventRecord(tev[k], s);
        if (L.items[c] == 0) continue;
        // with concurrency the first class stays on s, the others go to side streams
        cudaStream_t cs = conc && used > 0 ? side[used - 1] : s;
        used++;
        int blocks = std::max(1, (int)(g_cfg.batch_blocks[c] * T.grid_frac[c] + 0.5f));
        blocks = std::min(blocks, g_cfg.batch_blocks[c]);
        if (c == CLS_WARP) {
            const uint64_t warps = ((uint64_t)L.items[c] + B.warp_chunk - 1) / B.warp_chunk;
            blocks = (int)std::min<uint64_t>(blocks, (warps + WARP_THREADS / 32 - 1) / (WARP_THREADS / 32));
            k_warp_batch<<<blocks, WARP_THREADS, WARP_SMEM, cs>>>(B);
        } else {
            blocks = (int)std::min<uint64_t>(blocks, L.items[c]);
            if (c == CLS_TEAM) k_team_batch<<<blocks, TEAM_THREADS, TEAM_SMEM, cs>>>(B);
            else if (c == CLS_CTAH) k_ctah_batch<<<blocks, CTAH_THREADS, CTAH_SMEM, cs>>>(B);
            else k_dense_batch<<<blocks, DENSE_THREADS, DENSE_SMEM, cs>>>(B);
        }
        note_launch();
    }
    if (conc)
        for (int k = 0; k + 1 < used; k++) {
            cudaEventRecord(ev[1 + k], side[k]);
            cudaStreamWaitEvent(s, ev[1 + k], 0);
        }
    if (tev) cudaEventRecord(tev[NCLS], s);
    const uint32_t res_blocks = std::min<uint32_t>((L.n + 255) / 256, 1024);
    if (L.n) { k_batch_results<<<res_blocks, 256, 0, s>>>(B, L.out); note_launch(); }
}

void launch_flip(DevGraph &g, const int64_t *edge_idx_dev, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_flip<<<(unsigned)blocks, 256, 0, s>>>(g, edge_idx_dev, n); note_launch();
}

}  // namespace bb
