// walk.cuh - the wedge walkers and per-anchor helpers shared by the count
// kernels (count.cu) and the per-vertex / per-edge kernels (pervertex.cu).
//
// A walker streams the wedges of one anchor: for each of its middles v (the
// anchor's neighbours), a segment of v's row in the other side's adjacency
// (the endpoints u of the wedges anchor - v - u). The count kernels only
// add each wedge into its pair's tally; the per-vertex kernels walk a second
// time, reading the final tallies, and need each middle's sum of the values
// read (the "segment sums" of the walkers below).
#pragma once
#include <cstddef>
#include "graph.cuh"

namespace bb {
namespace walk {
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

// A chunk of middles, compacted to those with a non-empty segment, for the
// quad walker: the segment as a word range [st, en) of the middle side's
// adjacency (absolute, below 2^32 because nE is), the aligned 16-byte quads
// of the chunk before this segment (below 2^31) with the sign bit of the
// anchor's edge in bit 31, and the quads up to and including it.
struct alignas(16) QSeg {
    uint32_t st, en, excl_sw, incl;
};

template <int TS>
struct alignas(16) WalkSmem {
    QSeg seg[TS];
    unsigned long long warp_part[TS / 32];  // per warp: quads (low half), segments (high half)
    uint32_t tot[2];
};
// a lone warp scans with shuffles only
template <>
struct alignas(16) WalkSmem<32> {
    QSeg seg[32];
};

constexpr uint32_t EXMASK = 0x7fffffffu;

// aligned quads (four-entry, 16-byte blocks) that hold the words [st, st + len)
__device__ __forceinline__ uint32_t quads_of(uint32_t st, uint32_t len) {
    if (len == 0) return 0u;
    const uint32_t en = st + len;
    return (en >> 2) + ((en & 3u) != 0u) - (st >> 2);
}

// equal share t of n among TS threads
template <int TS>
__device__ __forceinline__ uint32_t share(uint32_t n, uint32_t t) {
    return (uint32_t)((unsigned long long)n * t / TS);
}

// Segment sums (second walks of the per-vertex kernels). With SUMS a
// walker's callback also gets the entry's absolute position in the middle
// side's adjacency and returns a u32 value (0 for an entry outside its
// segment); the walker adds the values of each segment into acc[k], k = the
// segment's compacted index in the chunk, and after the chunk hands every
// middle with a non-empty segment its sum: mid(j, sum) for the middle at
// index j of the anchor's row (sum may be 0). acc starts at zero and is left
// at zero. Every value summed per thread between flushes stays below 2^32.
struct NoMid {
    __device__ void operator()(uint32_t, unsigned long long) const {}
};

// Quad walker, per thread: the quads [a, b) of a compacted chunk (NZ
// segments). Every step loads whole aligned quads of the middle side's
// adjacency (one 16-byte load for four entries). A quad holds at least one
// entry of its segment, so it lies inside the adjacency's 16-byte-padded
// allocation. Threads get equal quad counts, so a team's lanes run the same
// number of steps. Entries outside a segment (in its first and last quad)
// are skipped: with BF, add(entry, vb, sign bit of the anchor's edge) is
// called for every entry with vb = 1 inside the segment and 0 outside
// (branch-free; add must then change nothing), otherwise add(entry, sign)
// is called for the entries inside only. Which form compiles to fewer
// instructions depends on the class (measured per class). SUMS (BF only):
// add(entry, vb, sign, position) returns the entry's value.
template <int U, bool BF, bool SUMS = false, typename Add>
__device__ __forceinline__ void quad_range(const uint4 *__restrict__ oadj4, const QSeg *seg,
                                           uint32_t NZ, uint32_t a, uint32_t b, Add &&add,
                                           unsigned long long *acc = nullptr) {
    static_assert(BF || !SUMS, "segment sums take the branch-free form");
    if (a >= b) return;
    uint32_t k = 0, hi = NZ;  // segment holding quad a: the first whose end is past a
    while (k < hi) {
        const uint32_t mid = (k + hi) >> 1;
        if (seg[mid].incl <= a) k = mid + 1; else hi = mid;
    }
    QSeg d = seg[k];
    uint32_t q = (d.st >> 2) + (a - (d.excl_sw & EXMASK));
    uint32_t qn = d.incl - a;  // quads left in this segment
    uint32_t kc = k, run = 0;  // SUMS: the running sum and its segment
    for (uint32_t i = a; i < b; i += U) {
        uint32_t qa[U], lo[U], hi4[U], sw[U], ku[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            lo[u] = 4u;  // an empty step: no entry passes lo <= j < hi4
            hi4[u] = 0u;
            qa[u] = 0u;
            sw[u] = 0u;
            if (i + u < b) {
                if (qn == 0) {
                    k++;
                    d = seg[k];
                    q = d.st >> 2;
                    qn = d.incl - (d.excl_sw & EXMASK);
                }
                const uint32_t w0 = q << 2;
                qa[u] = q;
                lo[u] = d.st > w0 ? d.st - w0 : 0u;
                hi4[u] = d.en - w0 < 4u ? d.en - w0 : 4u;
                sw[u] = d.excl_sw >> 31;
                q++;
                qn--;
            }
            ku[u] = k;
        }
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            v[u] = hi4[u] ? __ldg(oadj4 + qa[u]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < U; u++) {
            if constexpr (SUMS) {
                const uint32_t p = qa[u] << 2;
                const uint32_t s = add(v[u].x, (uint32_t)(lo[u] == 0u), sw[u], p) +
                                   add(v[u].y, (uint32_t)(lo[u] <= 1u && hi4[u] >= 2u), sw[u], p + 1) +
                                   add(v[u].z, (uint32_t)(lo[u] <= 2u && hi4[u] >= 3u), sw[u], p + 2) +
                                   add(v[u].w, (uint32_t)(hi4[u] == 4u), sw[u], p + 3);
                if (ku[u] != kc) {
                    if (run) atomicAdd(&acc[kc], (unsigned long long)run);
                    kc = ku[u];
                    run = 0;
                }
                run += s;
            } else if constexpr (BF) {
                add(v[u].x, (uint32_t)(lo[u] == 0u), sw[u]);
                add(v[u].y, (uint32_t)(lo[u] <= 1u && hi4[u] >= 2u), sw[u]);
                add(v[u].z, (uint32_t)(lo[u] <= 2u && hi4[u] >= 3u), sw[u]);
                add(v[u].w, (uint32_t)(hi4[u] == 4u), sw[u]);
            } else {
                if (lo[u] == 0u) add(v[u].x, sw[u]);
                if (lo[u] <= 1u && hi4[u] >= 2u) add(v[u].y, sw[u]);
                if (lo[u] <= 2u && hi4[u] >= 3u) add(v[u].z, sw[u]);
                if (hi4[u] == 4u) add(v[u].w, sw[u]);
            }
        }
    }
    if constexpr (SUMS)
        if (run) atomicAdd(&acc[kc], (unsigned long long)run);
}

// the same over [a, b) in sub-ranges of at most `span` quads, calling
// flush() after each (callers whose per-thread running sums must be
// bounded between flushes)
template <int U, bool BF, bool SUMS = false, typename Add, typename Flush>
__device__ __forceinline__ void quad_range_flushed(const uint4 *__restrict__ oadj4,
                                                   const QSeg *seg, uint32_t NZ, uint32_t a,
                                                   uint32_t b, uint32_t span, Add &&add,
                                                   Flush &&flush,
                                                   unsigned long long *acc = nullptr) {
    for (uint32_t s = a; s < b;) {
        const uint32_t e = b - s > span ? s + span : b;
        quad_range<U, BF, SUMS>(oadj4, seg, NZ, s, e, add, acc);
        flush();
        s = e;
    }
}

// One chunk of up to TS middles (j = this thread's middle, valid below m1):
// reads each middle's descriptor, takes its segment, and compacts the
// non-empty segments into sm.seg with their prefix in quads (QUADS) or in
// wedges. T = the chunk's quads or wedges, NZ = its segments (the same in
// every thread of the team), mine = the compacted index of this thread's
// segment (~0 when it is empty).
template <int TS, bool QUADS = true, typename Seg>
__device__ __forceinline__ void chunk_scan(const uint4 *__restrict__ smd, int64_t rb, uint32_t j,
                                           uint32_t m1, WalkSmem<TS> &sm, int t, Seg &&seg,
                                           uint32_t &T, uint32_t &NZ, uint32_t &mine) {
    const int lane = t & 31, w = t >> 5;
    long long st = 0;
    uint32_t len = 0, sw = 0;
    if (j < m1) {
        const uint4 d = smd[rb + j];
        sw = d.w;
        seg(d, st, len);
    }
    const uint32_t nq = QUADS ? quads_of((uint32_t)st, len) : len;
    uint32_t x = warp_incl_scan(nq);
    const unsigned nzb = __ballot_sync(FULL, nq > 0);
    uint32_t nzi = __popc(nzb & ((2u << lane) - 1u));
    if constexpr (TS > 32) {
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
    mine = nq > 0 ? nzi - 1 : ~0u;
    if (nq > 0) sm.seg[nzi - 1] = QSeg{(uint32_t)st, (uint32_t)st + len, (x - nq) | (sw << 31), x};
    if constexpr (TS == 32) {
        T = __shfl_sync(FULL, x, 31);
        NZ = __popc(nzb);
        __syncwarp();
    } else {
        if (t == TS - 1) { sm.tot[0] = x; sm.tot[1] = nzi; }
        team_sync<TS>();
        T = sm.tot[0];
        NZ = sm.tot[1];
    }
}

template <int TS, bool QUADS = true, typename Seg>
__device__ __forceinline__ void chunk_scan(const uint4 *__restrict__ smd, int64_t rb, uint32_t j,
                                           uint32_t m1, WalkSmem<TS> &sm, int t, Seg &&seg,
                                           uint32_t &T, uint32_t &NZ) {
    uint32_t mine;
    chunk_scan<TS, QUADS>(smd, rb, j, m1, sm, t, seg, T, NZ, mine);
}

// After a chunk walked with segment sums: each thread takes its segment's
// sum (and resets it) and hands it to mid.
template <int TS, typename Acc, typename Mid>
__device__ __forceinline__ void chunk_sums(Acc *acc, uint32_t mine, uint32_t j, Mid &&mid) {
    team_sync<TS>();
    if (mine != ~0u) {
        const unsigned long long s = acc[mine];
        acc[mine] = 0;
        mid(j, s);
    }
}

// Walk the wedges of one anchor's middles [m0, m1) (its row starts at rb in
// the anchor side's descriptors smd; the middles' rows are in oadj) as a
// team of TS threads (t = thread index in the team): per chunk of TS
// middles, a chunk scan and then each thread's equal share of the chunk's
// quads. seg(md, st, len) picks the segment [st, st+len) of a middle's row
// from its descriptor; add is called as in quad_range, once per wedge
// (entry = endpoint side rank << 1 | sign of the middle-endpoint edge).
// flush() follows every `span` quads of a thread. SUMS: segment sums into
// acc (TS entries), handed to mid per chunk.
template <int TS, int U, bool BF, bool SUMS = false, typename Seg, typename Add, typename Flush,
          typename Mid = NoMid>
__device__ __forceinline__ void quad_walk(const uint4 *__restrict__ smd,
                                          const uint32_t *__restrict__ oadj, int64_t rb,
                                          uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                          uint32_t span, Seg &&seg, Add &&add, Flush &&flush,
                                          unsigned long long *acc = nullptr, Mid &&mid = Mid{}) {
    const uint4 *oadj4 = reinterpret_cast<const uint4 *>(oadj);
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ, mine;
        chunk_scan<TS>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ, mine);
        quad_range_flushed<U, BF, SUMS>(oadj4, sm.seg, NZ, share<TS>(T, t),
                                        share<TS>(T, t + 1), span, add, flush, acc);
        if constexpr (SUMS) chunk_sums<TS>(acc, mine, mc + (uint32_t)t, mid);
        team_sync<TS>();
    }
}

// Lanes of a warp round that share a segment: the round's positions are
// consecutive, so a segment's lanes are consecutive too. M has bit s set
// when a segment starts at the round's position s; lanes at or past
// `valid` hold no position. Returns the lanes of this lane's segment
// (within the valid ones); head = the segment's first lane in the round.
__device__ __forceinline__ unsigned round_peers(unsigned M, uint32_t lane, uint32_t valid,
                                                bool &head) {
    const unsigned upto = (2u << lane) - 1u;
    const unsigned Mh = M | 1u;  // lane 0 heads its segment in any round
    const uint32_t h = 31u - __clz(Mh & upto);
    const unsigned above = Mh & ~upto;
    const unsigned below_next = above ? (above & (0u - above)) - 1u : FULL;
    const unsigned vmask = valid >= 32u ? FULL : (1u << valid) - 1u;
    head = lane == h;
    return below_next & (FULL << h) & vmask;
}

// Where a lane's quad or wedge of a round sits, for segment sums: its
// segment's compacted index k, the lanes sharing that segment in the round
// (round_peers) and the entry position p (of the quad's first entry).
struct RoundPos {
    uint32_t k = 0, p = 0;
    unsigned peers = 0;
    bool head = false;
};

// Team walker in coalesced rounds. After the chunk scan each warp of the
// team takes an equal part [A, B) of the chunk's quads and walks it in
// rounds of 32 consecutive quads, lane l taking quad r + l (a round reads
// up to 512 consecutive bytes of a segment). The segments that start inside
// a round are found from the next 32 compacted segments, one per lane, whose
// starts form a bitmask (one warp OR-reduction); a lane's segment is the
// last one starting at or before its quad. Each round's quads are loaded one
// round ahead. add is called as in quad_range (BF chooses the form);
// flush() follows every `span` rounds of a warp and the end of its part.
// SUMS (BF only): add(entry, vb, sign, position) returns the entry's value;
// a round's values are summed per segment across its lanes (one warp
// reduction) and added into acc (TS entries, u32 or u64 as the caller's
// sums need), handed to mid per chunk.
template <int TS, bool BF, bool SUMS = false, typename Seg, typename Add, typename Flush,
          typename Mid = NoMid, typename Acc = unsigned long long>
__device__ __forceinline__ void team_rounds(const uint4 *__restrict__ smd,
                                            const uint32_t *__restrict__ oadj, int64_t rb,
                                            uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                            uint32_t span, Seg &&seg, Add &&add, Flush &&flush,
                                            Acc *acc = nullptr, Mid &&mid = Mid{}) {
    static_assert(BF || !SUMS, "segment sums take the branch-free form");
    constexpr uint32_t NW = TS / 32;
    const uint4 *oadj4 = reinterpret_cast<const uint4 *>(oadj);
    const uint32_t lane = (uint32_t)t & 31u, w = (uint32_t)t >> 5;
    const unsigned upto = (2u << lane) - 1u;
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ, mine;
        chunk_scan<TS>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ, mine);
        const uint32_t A = share<NW>(T, w), B = share<NW>(T, w + 1);
        if (A < B) {
            uint32_t kb = 0, hi = NZ;  // segment holding quad A
            while (kb < hi) {
                const uint32_t mid = (kb + hi) >> 1;
                if (sm.seg[mid].incl <= A) kb = mid + 1; else hi = mid;
            }
            kb++;  // next segment to start
            // lane's quad of the round at r: loads it, sets vm (0 past B) and sw
            auto locate = [&](uint32_t r, uint4 &v, uint32_t &vm, uint32_t &swq, RoundPos &pos) {
                const uint32_t c = kb + lane;
                const uint32_t s = c < NZ ? (sm.seg[c].excl_sw & EXMASK) - r : 32u;
                const unsigned M = __reduce_or_sync(FULL, s < 32u ? 1u << s : 0u);
                const uint32_t k = kb - 1u + __popc(M & upto);
                kb += __popc(M);
                const uint32_t q = r + lane;
                vm = 0u;
                if constexpr (SUMS) {
                    pos.k = k;
                    pos.peers = round_peers(M, lane, B - r, pos.head);
                }
                if (q < B) {
                    const QSeg d = sm.seg[k];
                    const uint32_t qq = (d.st >> 2) + (q - (d.excl_sw & EXMASK));
                    const uint32_t w0 = qq << 2;
                    const uint32_t lo = d.st > w0 ? d.st - w0 : 0u;
                    const uint32_t hq = d.en - w0 < 4u ? d.en - w0 : 4u;
                    vm = (0xfu >> (4u - hq)) & (0xfu << lo);
                    swq = d.excl_sw >> 31;
                    pos.p = w0;
                    v = __ldg(oadj4 + qq);
                }
            };
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            uint32_t vm = 0u, swq = 0u, rounds = 0u;
            RoundPos pos;
            locate(A, v, vm, swq, pos);
            for (uint32_t r = A; r < B; r += 32) {
                uint4 vn = make_uint4(0u, 0u, 0u, 0u);
                uint32_t vmn = 0u, swn = 0u;
                RoundPos posn;
                if (r + 32 < B) locate(r + 32, vn, vmn, swn, posn);
                if constexpr (SUMS) {
                    if (vm) {  // the round's valid lanes (a prefix of the warp)
                        const uint32_t val = add(v.x, vm & 1u, swq, pos.p) +
                                             add(v.y, (vm >> 1) & 1u, swq, pos.p + 1) +
                                             add(v.z, (vm >> 2) & 1u, swq, pos.p + 2) +
                                             add(v.w, vm >> 3, swq, pos.p + 3);
                        const uint32_t tot = __reduce_add_sync(pos.peers, val);
                        if (pos.head && tot) atomicAdd(&acc[pos.k], (Acc)tot);
                    }
                } else if constexpr (BF) {
                    add(v.x, vm & 1u, swq);
                    add(v.y, (vm >> 1) & 1u, swq);
                    add(v.z, (vm >> 2) & 1u, swq);
                    add(v.w, vm >> 3, swq);
                } else {
                    if (vm & 1u) add(v.x, swq);
                    if (vm & 2u) add(v.y, swq);
                    if (vm & 4u) add(v.z, swq);
                    if (vm & 8u) add(v.w, swq);
                }
                v = vn;
                vm = vmn;
                swq = swn;
                pos = posn;
                if (++rounds == span) { flush(); rounds = 0u; }
            }
            flush();
        }
        if constexpr (SUMS) chunk_sums<TS>(acc, mine, mc + (uint32_t)t, mid);
        team_sync<TS>();
    }
}

// Wedge walker, per thread: the wedges [a, b) of a compacted chunk whose
// prefix is in wedges, U loads in flight per step, one(entry, sign bit of
// the anchor's edge) per wedge. For segment families whose per-wedge work
// is a loop (hash probes): one call site, no predicated quad entries.
// SUMS: one(entry, sign, position) returns the wedge's value, summed per
// segment into acc.
template <int U, bool SUMS = false, typename One>
__device__ __forceinline__ void wedge_range(const uint32_t *__restrict__ oadj, const QSeg *seg,
                                            uint32_t NZ, uint32_t a, uint32_t b, One &&one,
                                            unsigned long long *acc = nullptr) {
    if (a >= b) return;
    uint32_t k = 0, hi = NZ;  // segment holding wedge a
    while (k < hi) {
        const uint32_t mid = (k + hi) >> 1;
        if (seg[mid].incl <= a) k = mid + 1; else hi = mid;
    }
    QSeg d = seg[k];
    uint32_t p = d.st + (a - (d.excl_sw & EXMASK));
    uint32_t kc = k, run = 0;  // SUMS: the running sum and its segment
    for (uint32_t i = a; i < b; i += U) {
        uint32_t pa[U], sq[U], ku[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            pa[u] = 0xffffffffu;
            sq[u] = 0u;
            if (i + u < b) {
                if (p == d.en) {
                    k++;
                    d = seg[k];
                    p = d.st;
                }
                pa[u] = p++;
                sq[u] = d.excl_sw >> 31;
            }
            ku[u] = k;
        }
        uint32_t xv[U];
#pragma unroll
        for (int u = 0; u < U; u++) xv[u] = pa[u] != 0xffffffffu ? __ldg(oadj + pa[u]) : 0u;
        for (int u = 0; u < U; u++) {
            if (pa[u] == 0xffffffffu) continue;
            if constexpr (SUMS) {
                const uint32_t val = one(xv[u], sq[u], pa[u]);
                if (ku[u] != kc) {
                    if (run) atomicAdd(&acc[kc], (unsigned long long)run);
                    kc = ku[u];
                    run = 0;
                }
                run += val;
            } else {
                one(xv[u], sq[u]);
            }
        }
    }
    if constexpr (SUMS)
        if (run) atomicAdd(&acc[kc], (unsigned long long)run);
}

// quad_walk's counterpart over wedges (wedge_range per thread)
template <int TS, int U, bool SUMS = false, typename Seg, typename One, typename Flush,
          typename Mid = NoMid>
__device__ __forceinline__ void wedge_walk(const uint4 *__restrict__ smd,
                                           const uint32_t *__restrict__ oadj, int64_t rb,
                                           uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                           uint32_t span, Seg &&seg, One &&one, Flush &&flush,
                                           unsigned long long *acc = nullptr, Mid &&mid = Mid{}) {
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ, mine;
        chunk_scan<TS, false>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ, mine);
        const uint32_t a = share<TS>(T, t), b = share<TS>(T, t + 1);
        for (uint32_t s0 = a; s0 < b;) {
            const uint32_t e = b - s0 > span ? s0 + span : b;
            wedge_range<U, SUMS>(oadj, sm.seg, NZ, s0, e, one, acc);
            flush();
            s0 = e;
        }
        if constexpr (SUMS) chunk_sums<TS>(acc, mine, mc + (uint32_t)t, mid);
        team_sync<TS>();
    }
}

// One warp walks two segment families of an anchor's middles (the
// hub-window part and the part below it) from one chunk scan per 32
// middles, in rounds. A round of the first family covers 32 consecutive
// quads of the chunk's compacted quad range, lane l taking quad r + l, so
// the lanes of a round read consecutive quads of a segment (coalesced
// 16-byte loads); a round of the second family covers 32 consecutive
// wedges, one per lane. A lane finds the segment of its quad or wedge from
// the bitmask of the segments that start inside the round (one warp
// OR-reduction): it is the last segment starting at or before its
// position. quada(v, vm, sw) takes a loaded quad (vm: its entries inside
// the segment, bit j for entry j; the quad is only read when vm != 0) and
// oneb(x, sw, valid) one wedge of the second family; sw is the sign bit of
// the anchor's edge to the middle. The second family's first round calls
// oneb on every lane of the warp (valid = false: no wedge on this lane), so
// that oneb may use warp-wide operations when that round is the only one
// (at most 32 wedges in the chunk); later rounds call it on valid lanes.
//
// SUMS: quada(v, vm, sw, p) and oneb(x, sw, p) also get the position p of
// the quad's first entry or of the wedge and return a value; the values of
// each segment are summed (one warp reduction per round over the lanes
// sharing a segment) into acc (64 u32 entries: the first family's segments,
// then the second's), and after each chunk mid(j, sum) is called for every
// middle j with a non-empty segment in either family.
template <bool SUMS = false, typename SegA, typename QuadA, typename SegB, typename OneB,
          typename Mid = NoMid>
__device__ __forceinline__ void warp_rounds(const uint4 *__restrict__ smd,
                                            const uint32_t *__restrict__ oadj, int64_t rb,
                                            uint32_t m0, uint32_t m1, WalkSmem<32> &sa,
                                            WalkSmem<32> &sb, unsigned lane, SegA &&sega,
                                            QuadA &&quada, SegB &&segb, OneB &&oneb,
                                            uint32_t *acc = nullptr, Mid &&mid = Mid{}) {
    const uint4 *oadj4 = reinterpret_cast<const uint4 *>(oadj);
    const unsigned upto = (2u << lane) - 1u;
    for (uint32_t mc = m0; mc < m1; mc += 32) {
        const uint32_t j = mc + lane;
        long long sta = 0, stb = 0;
        uint32_t la = 0, lb = 0, sw = 0;
        if (j < m1) {
            const uint4 d = smd[rb + j];
            sw = d.w;
            sega(d, sta, la);
            segb(d, stb, lb);
        }
        // one scan of both families' sizes in 16-bit halves: an anchor of
        // the warp class has at most WARP_W_MAX wedges, so neither sum wraps
        static_assert(WARP_W_MAX < 0xffff, "packed warp chunk scan");
        const uint32_t qa = quads_of((uint32_t)sta, la);
        const uint32_t x = warp_incl_scan(qa | (lb << 16));
        const uint32_t xa = x & 0xffffu, xb = x >> 16;
        const uint32_t ea = xa - qa, eb = xb - lb;  // first quad / wedge of this lane's segments
        const unsigned nza = __ballot_sync(FULL, qa > 0), nzb = __ballot_sync(FULL, lb > 0);
        const uint32_t ka = __popc(nza & upto) - 1u, kbm = __popc(nzb & upto) - 1u;
        if (qa > 0) sa.seg[ka] = QSeg{(uint32_t)sta, (uint32_t)sta + la, ea | (sw << 31), xa};
        if (lb > 0) sb.seg[kbm] = QSeg{(uint32_t)stb, (uint32_t)stb + lb, eb | (sw << 31), xb};
        const uint32_t TA = __shfl_sync(FULL, xa, 31), TB = __shfl_sync(FULL, xb, 31);
        __syncwarp();
        // The second family's first round is loaded before the first
        // family's rounds run, and each round of the first family loads its
        // quads one round ahead: a warp keeps two loads in flight instead of
        // waiting out one memory round trip per round.
        uint32_t xb0 = 0, swb0 = 0, baseb = 0;
        bool hb0 = false;
        RoundPos posb0;
        if (TB > 0) {
            const unsigned M = __reduce_or_sync(FULL, (lb > 0 && eb < 32u) ? 1u << eb : 0u);
            const uint32_t k = __popc(M & upto) - 1u;
            baseb = __popc(M);
            if constexpr (SUMS) {
                posb0.k = k;
                posb0.peers = round_peers(M, lane, TB, posb0.head);
            }
            if (lane < TB) {
                const QSeg d = sb.seg[k];
                posb0.p = d.st + (lane - (d.excl_sw & EXMASK));
                xb0 = oadj[posb0.p];
                swb0 = d.excl_sw >> 31;
                hb0 = true;
            }
        }
        // a round's values, summed over the lanes of each segment; valid
        // lanes only (a prefix of the warp)
        auto round_sum = [&](uint32_t val, const RoundPos &pos, uint32_t off) {
            const uint32_t tot = __reduce_add_sync(pos.peers, val);
            if (pos.head && tot) atomicAdd(&acc[off + pos.k], tot);
        };
        uint32_t base = 0;  // segments of the first family starting before the next round
        // quad of lane `lane` in the round starting at quad r: loads it and
        // sets vm (0 past the chunk's quads) and sw
        auto locate = [&](uint32_t r, uint4 &v, uint32_t &vm, uint32_t &swq, RoundPos &pos) {
            const uint32_t s = ea - r;
            const unsigned M = __reduce_or_sync(FULL, (qa > 0 && s < 32u) ? 1u << s : 0u);
            const uint32_t k = base + __popc(M & upto) - 1u;
            base += __popc(M);
            const uint32_t q = r + lane;
            vm = 0u;
            if constexpr (SUMS) {
                pos.k = k;
                pos.peers = round_peers(M, lane, TA - r, pos.head);
            }
            if (q < TA) {
                const QSeg d = sa.seg[k];
                const uint32_t qq = (d.st >> 2) + (q - (d.excl_sw & EXMASK));
                const uint32_t w0 = qq << 2;
                const uint32_t lo = d.st > w0 ? d.st - w0 : 0u;
                const uint32_t hi = d.en - w0 < 4u ? d.en - w0 : 4u;
                vm = (0xfu >> (4u - hi)) & (0xfu << lo);
                swq = d.excl_sw >> 31;
                pos.p = w0;
                v = __ldg(oadj4 + qq);
            }
        };
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        uint32_t vm = 0u, swq = 0u;
        RoundPos pos;
        if (TA > 0) locate(0, v, vm, swq, pos);
        for (uint32_t r = 0; r < TA; r += 32) {
            uint4 vn = make_uint4(0u, 0u, 0u, 0u);
            uint32_t vmn = 0u, swn = 0u;
            RoundPos posn;
            if (r + 32 < TA) locate(r + 32, vn, vmn, swn, posn);
            if constexpr (SUMS) {
                if (vm) round_sum(quada(v, vm, swq, pos.p), pos, 0u);
            } else {
                if (vm) quada(v, vm, swq);
            }
            v = vn;
            vm = vmn;
            swq = swn;
            pos = posn;
        }
        if constexpr (SUMS) {
            if (hb0) round_sum(oneb(xb0, swb0, posb0.p), posb0, 32u);
        } else {
            if (TB > 0) oneb(xb0, swb0, hb0);
        }
        for (uint32_t r = 32; r < TB; r += 32) {
            const uint32_t s = eb - r;
            const unsigned M = __reduce_or_sync(FULL, (lb > 0 && s < 32u) ? 1u << s : 0u);
            const uint32_t k = baseb + __popc(M & upto) - 1u;
            baseb += __popc(M);
            const uint32_t p = r + lane;
            if (p < TB) {
                const QSeg d = sb.seg[k];
                const uint32_t e = d.st + (p - (d.excl_sw & EXMASK));
                if constexpr (SUMS) {
                    RoundPos pb;
                    pb.k = k;
                    pb.peers = round_peers(M, lane, TB - r, pb.head);
                    round_sum(oneb(oadj[e], d.excl_sw >> 31, e), pb, 32u);
                } else {
                    oneb(oadj[e], d.excl_sw >> 31, true);
                }
            }
        }
        __syncwarp();
        if constexpr (SUMS) {
            uint32_t sum = 0;
            if (qa > 0) { sum += acc[ka]; acc[ka] = 0u; }
            if (lb > 0) { sum += acc[32 + kbm]; acc[32 + kbm] = 0u; }
            if (qa > 0 || lb > 0) mid(j, sum);
            __syncwarp();
        }
    }
}

// Open-addressing tables in shared memory of 2^(32-shift) u64 slots: the
// key (endpoint + 1; 0 = empty) in the high half and the packed tallies
// (S | A << 16) in the low half. hash_add inserts or finds the key and adds
// inc to its tallies (an insert sets key and first tally in one
// compare-and-swap); it returns the tallies the key held before.
// CAS_FIRST tries the insert before any read of the slot (most keys of the
// hashed endpoints are new; a slot that holds the key then takes the add);
// otherwise the slot is read first. Both give the same result.
template <bool CAS_FIRST = true>
__device__ __forceinline__ uint32_t hash_add(unsigned long long *tab, uint32_t shift,
                                             uint32_t mask, uint32_t key, uint32_t inc,
                                             uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    const unsigned long long want = ((unsigned long long)key << 32) | inc;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        if constexpr (CAS_FIRST) {
            const unsigned long long old = atomicCAS(&tab[h], 0ull, want);
            if (old == 0ull) return 0u;
            if ((uint32_t)(old >> 32) == key)
                return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
        } else {
            const unsigned long long cur = *((volatile unsigned long long *)&tab[h]);
            const uint32_t k = (uint32_t)(cur >> 32);
            if (k == key) return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
            if (k == 0) {
                const unsigned long long old = atomicCAS(&tab[h], 0ull, want);
                if (old == 0ull) return 0u;
                if ((uint32_t)(old >> 32) == key)
                    return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
            }
        }
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
    return 0u;
}

// the packed tallies a key holds (read-only probe of a filled table); a
// missing key is an internal error
__device__ __forceinline__ uint32_t hash_find(const unsigned long long *tab, uint32_t shift,
                                              uint32_t mask, uint32_t key, uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const unsigned long long cur = tab[h];
        if ((uint32_t)(cur >> 32) == key) return (uint32_t)cur;
        if (cur == 0ull) break;
        h = (h + 1) & mask;
    }
    set_error(err, E_PROBE);
    return 0u;
}

// Running sums of one thread, per wedge: own += the previous value of the
// wedge's own tally, other += the previous value of the pair's other tally.
// Over all wedges own is the balanced count (C(S,2) + C(A,2) per pair) and
// own + other the total (C(S+A,2)). dp2a picks a 16-bit half of the packed
// tallies by a byte mask: 1 for S, 0x100 for A.
template <bool CAS_FIRST = true>
__device__ __forceinline__ void hash_wedge32(unsigned long long *tab, uint32_t shift,
                                             uint32_t mask, uint32_t x, uint32_t sw,
                                             uint32_t *err, uint32_t &own, uint32_t &other) {
    const uint32_t asym = (x ^ sw) & 1u;
    const uint32_t old =
        hash_add<CAS_FIRST>(tab, shift, mask, (x >> 1) + 1, asym ? INC_ASYM : INC_SYM, err);
    const uint32_t pick = 1u << (asym << 3);
    own = __dp2a_lo(old, pick, own);
    other = __dp2a_lo(old, pick ^ 0x0101u, other);
}

// One round of at most 32 wedges of an anchor (all lanes of the warp call
// it; valid = false: no wedge on this lane), counted without a table: the
// lanes holding the same endpoint are found by one warp match, and a
// wedge's previous tallies are the matching wedges on lower lanes of its
// own and of the other type (the same sums as hash_wedge32, for wedges
// taken in lane order).
__device__ __forceinline__ void match_wedges(uint32_t x, uint32_t sw, bool valid, uint32_t lane,
                                             uint32_t &own, uint32_t &other) {
    const unsigned vmask = __ballot_sync(FULL, valid);
    const unsigned m = __match_any_sync(FULL, valid ? (x >> 1) : 0xffffffffu) & vmask;
    const uint32_t asym = (x ^ sw) & 1u;
    const unsigned B = __ballot_sync(FULL, asym);
    const unsigned same = m & (asym ? B : ~B);
    const unsigned lower = (1u << lane) - 1u;
    if (valid) {
        own += __popc(same & lower);
        other += __popc(m & ~same & lower);
    }
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
// hash for endpoints below the window, and the walker's chunks.
//
// The hub window holds the top HUB_WINDOW side ranks; a rank's counter is
// at rank mod HUB_WINDOW, one to one on any HUB_WINDOW consecutive ranks.
// With entry x = rank << 1 | sign: the counter's word is at byte offset
// x & (2 HUB_WINDOW - 4), its half is bit 1 of x, and bit 0 of x xor the
// anchor edge's sign picks the byte (S or A).
struct alignas(16) WarpSmem {
    uint32_t win[HUB_WINDOW / 2];
    unsigned long long tab[WARP_CAP];
    WalkSmem<32> walk, walk2;  // hub-window and below-window segments
};

// per-warp copies are laid out back to back and reset with 16-byte stores
static_assert(sizeof(WarpSmem) % 16 == 0, "WarpSmem must keep 16-byte alignment");
static_assert((HUB_WINDOW & (HUB_WINDOW - 1)) == 0, "hub window indexes are masked");
static_assert(offsetof(WarpSmem, tab) % 16 == 0, "table needs 16-byte alignment");

// the side rank whose hub-window counter is at index i (rank mod
// HUB_WINDOW): the window holds ranks [wb, wb + HUB_WINDOW)
__device__ __forceinline__ uint32_t window_rank(uint32_t i, uint32_t wb) {
    return wb + ((i - wb) & (HUB_WINDOW - 1u));
}

// first rank of the hub window of a side of ns vertices
__device__ __forceinline__ uint32_t window_base(int64_t ns) {
    return ns > (int64_t)HUB_WINDOW ? (uint32_t)(ns - HUB_WINDOW) : 0u;
}

// What a warp-class anchor's tally pass leaves in shared memory: whether
// the hub window holds counts, and the hash table's geometry (cap = 0: no
// table).
struct WarpTab {
    uint32_t cap = 0, shift = 0;
    bool hub = false;
};

// The tally pass of one warp-class anchor, walked by one warp: every wedge
// adds 1 to its pair's tally, own += the previous value of that tally and
// other += the previous value of the pair's other tally (per lane).
// MATCH: an anchor of at most 32 middles whose hashed wedges number at most
// 32 (one round) counts them by warp matching and keeps no table (its
// WarpTab has cap = 0); without MATCH every hashed wedge is in the table.
template <bool MATCH = false>
__device__ __forceinline__ WarpTab warp_tally(const DevGraph &G, WarpSmem &sm,
                                              const AnchorRec &rec, const Anchor &A,
                                              unsigned lane, uint32_t &own, uint32_t &other) {
    uint32_t *err = &G.scratch->err;
    const uint64_t W = A.W, above = (uint64_t)(A.ns - A.r - 1);
    WarpTab tb;
    // 32-bit sums: an anchor has at most WARP_W_MAX wedges, each adding less
    // than 2^8 to each sum (tallies are bounded by the degree <= WARP_DEG_MAX)
    static_assert(WARP_W_MAX * WARP_DEG_MAX < (1ull << 32), "32-bit warp sums");
    auto none = [](const uint4 &, long long &st, uint32_t &len) { st = 0; len = 0; };
    auto no_quad = [](const uint4 &, uint32_t, uint32_t) {};
    if (rec.flags & REC_HASH_ALL) {  // hash every endpoint
        const bool small = MATCH && A.deg <= 32u && W <= 32u;
        if (!small) table_geometry(W < above ? W : above, 32, WARP_CAP, tb.cap, tb.shift);
        const uint32_t mask = tb.cap - 1, shift = tb.shift;
        warp_rounds(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, lane, none, no_quad,
                    FullSeg{}, [&](uint32_t x, uint32_t sw, bool valid) {
                        if (small) match_wedges(x, sw, valid, lane, own, other);
                        else if (valid) hash_wedge32(sm.tab, shift, mask, x, sw, err, own, other);
                    });
    } else {
        tb.hub = true;
        const uint32_t wb = window_base(A.ns);
        const uint64_t wnh = A.wnh;
        const uint64_t above_nh = wb > A.r + 1 ? (uint64_t)wb - A.r - 1 : 0;
        const bool small = MATCH && A.deg <= 32u && wnh <= 32u;
        if (wnh > 0 && !small)
            table_geometry(wnh < above_nh ? wnh : above_nh, 32, WARP_CAP, tb.cap, tb.shift);
        const uint32_t mask = tb.cap - 1, shift = tb.shift;
        char *win = reinterpret_cast<char *>(sm.win);
        // one hub-window wedge (vb = 1) or an entry of the quad outside the
        // segment (vb = 0: adds 0 and picks nothing); the increment is the
        // tally byte's lowest bit, and as a dp4a byte mask it picks that
        // tally's previous value out of the returned word (the other
        // tally's byte for `other`)
        auto hub_one = [&](uint32_t x, uint32_t vb, uint32_t sw) {
            const uint32_t sh = ((x ^ sw) & 3u) << 3;
            const uint32_t inc = vb << sh;
            const uint32_t old =
                atomicAdd(reinterpret_cast<uint32_t *>(win + (x & (2u * HUB_WINDOW - 4u))), inc);
            own = __dp4a(old, inc, own);
            other = __dp4a(old, __byte_perm(inc, 0u, 0x2301u), other);  // the half's other byte
        };
        warp_rounds(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, lane, HubSeg{},
                    [&](const uint4 &v, uint32_t vm, uint32_t sw) {
                        hub_one(v.x, vm & 1u, sw);
                        hub_one(v.y, (vm >> 1) & 1u, sw);
                        hub_one(v.z, (vm >> 2) & 1u, sw);
                        hub_one(v.w, vm >> 3, sw);
                    },
                    LowSeg{}, [&](uint32_t x, uint32_t sw, bool valid) {
                        if (small) match_wedges(x, sw, valid, lane, own, other);
                        else if (valid) hash_wedge32(sm.tab, shift, mask, x, sw, err, own, other);
                    });
    }
    return tb;
}

__device__ __forceinline__ WarpSmem &warp_smem_init(unsigned char *smem_raw, unsigned lane,
                                                    size_t stride = sizeof(WarpSmem)) {
    WarpSmem &sm = *reinterpret_cast<WarpSmem *>(smem_raw + (threadIdx.x >> 5) * stride);
    clear_table<32>(sm.tab, WARP_CAP, (int)lane);
    for (uint32_t i = lane; i < HUB_WINDOW / 2; i += 32) sm.win[i] = 0u;
    __syncwarp();
    return sm;
}

// ------------------------------------------------- team and CTA-hash classes
// Per CTA: the hub window as 32-bit counters (S | A << 16) at rank mod
// HUB_WINDOW, a hash for endpoints below the window, and the walker's chunk.
template <int TS, uint32_t HCAP>
struct alignas(16) HybSmem {
    uint32_t win[HUB_WINDOW];             // hub window counters
    unsigned long long tab[HCAP];         // hash for endpoints below the window
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

// Running sums in 32 bits: a wedge adds its pair's previous tallies, which
// are at most the anchor's degree (<= MAX_DEGREE), so SUM_SPAN quads of one
// thread (four wedges each) cannot wrap a u32 before the walker flushes
// them into the 64-bit sums.
constexpr uint32_t SUM_SPAN = 8192;
static_assert((unsigned long long)SUM_SPAN * 4 * MAX_DEGREE < (1ull << 32), "32-bit span sums");

// quads per thread step of the hybrid classes' hub walks (per-thread quad
// shares measured faster than warp rounds for these classes)
template <int TS>
constexpr int HYBRID_QUADS = TS == TEAM_THREADS ? 1 : 2;

// what a hybrid anchor's tally pass leaves: hub window used, hash geometry
struct HybTab {
    uint32_t cap = 0, shift = 0;
    bool hub = false;
};

// The tally pass of one team/CTA-hash anchor, walked by the whole CTA; adds
// each thread's part of the anchor's balanced and total counts to bal, tot.
// CAS_FIRST: as in hash_add (the per-vertex kernels keep the read-first
// insert, which compiles to fewer registers in their larger bodies).
template <int TS, uint32_t HCAP, bool CAS_FIRST = true>
__device__ __forceinline__ HybTab hybrid_tally(const DevGraph &G, HybSmem<TS, HCAP> &sm,
                                               const Anchor &A, unsigned long long &bal,
                                               unsigned long long &tot) {
    const int t = threadIdx.x;
    uint32_t *err = &G.scratch->err;
    const uint32_t wb = window_base(A.ns);
    const uint64_t W = A.W, wnh = A.wnh;
    const uint64_t above_nh = wb > A.r + 1 ? (uint64_t)wb - A.r - 1 : 0;
    // hub walk: hb = the wedges' own previous tallies, ht = both previous
    // tallies; hash walk: own and other as in hash_wedge32
    constexpr int QU = HYBRID_QUADS<TS>;
    uint32_t hb = 0, ht = 0, own = 0, other = 0;
    auto flush = [&]() {
        bal += (unsigned long long)hb + own;
        tot += (unsigned long long)ht + own + other;
        hb = ht = own = other = 0;
    };
    HybTab tb;
    if (W > wnh) {  // endpoints inside the hub window
        tb.hub = true;
        // counter of a rank at rank mod HUB_WINDOW (one to one on the
        // window's consecutive ranks); an entry outside its segment (vb = 0)
        // adds 0 and picks nothing
        quad_walk<TS, QU, true>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, SUM_SPAN, HubSeg{},
                                [&](uint32_t x, uint32_t vb, uint32_t sw) {
                                    const uint32_t asym = (x ^ sw) & 1u;
                                    const uint32_t old =
                                        atomicAdd(&sm.win[(x >> 1) & (HUB_WINDOW - 1)],
                                                  vb << (asym << 4));
                                    hb = __dp2a_lo(old, vb << (asym << 3), hb);
                                    ht = __dp2a_lo(old, vb * 0x0101u, ht);
                                },
                                flush);
    }
    if (wnh > 0) {  // endpoints below the window
        table_geometry(wnh < above_nh ? wnh : above_nh, 32, HCAP, tb.cap, tb.shift);
        const uint32_t mask = tb.cap - 1, shift = tb.shift;
        wedge_walk<TS, 2>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, 4 * SUM_SPAN, LowSeg{},
                          [&](uint32_t x, uint32_t sw) {
                              hash_wedge32<CAS_FIRST>(sm.tab, shift, mask, x, sw, err, own,
                                                      other);
                          },
                          flush);
    }
    return tb;
}


}  // namespace walk
}  // namespace bb
