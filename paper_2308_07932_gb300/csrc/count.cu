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
// Work is spread by the quad walker: a team (a warp, or a whole CTA) loads a
// chunk of the anchor's middles, takes each middle's segment of the other
// side's adjacency, counts the aligned 16-byte quads that hold it and
// compacts the non-empty segments. Every thread then takes an equal share
// of the chunk's quads and streams through them, one 16-byte load per four
// entries, with the entries outside their segment predicated off.
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
//           Anchors of degree above MAX_DEGREE are wide jobs: 32-bit S and
//           A fields (u64 counters), one CTA each.
#include <algorithm>
#include <cstddef>
#include <mutex>
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
// instructions depends on the class (measured per class).
template <int U, bool BF, typename Add>
__device__ __forceinline__ void quad_range(const uint4 *__restrict__ oadj4, const QSeg *seg,
                                           uint32_t NZ, uint32_t a, uint32_t b, Add &&add) {
    if (a >= b) return;
    uint32_t k = 0, hi = NZ;  // segment holding quad a: the first whose end is past a
    while (k < hi) {
        const uint32_t mid = (k + hi) >> 1;
        if (seg[mid].incl <= a) k = mid + 1; else hi = mid;
    }
    QSeg d = seg[k];
    uint32_t q = (d.st >> 2) + (a - (d.excl_sw & EXMASK));
    uint32_t qn = d.incl - a;  // quads left in this segment
    for (uint32_t i = a; i < b; i += U) {
        uint32_t qa[U], lo[U], hi4[U], sw[U];
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
        }
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            v[u] = hi4[u] ? __ldg(oadj4 + qa[u]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < U; u++) {
            if constexpr (BF) {
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
}

// the same over [a, b) in sub-ranges of at most `span` quads, calling
// flush() after each (callers whose per-thread running sums must be
// bounded between flushes)
template <int U, bool BF, typename Add, typename Flush>
__device__ __forceinline__ void quad_range_flushed(const uint4 *__restrict__ oadj4,
                                                   const QSeg *seg, uint32_t NZ, uint32_t a,
                                                   uint32_t b, uint32_t span, Add &&add,
                                                   Flush &&flush) {
    for (uint32_t s = a; s < b;) {
        const uint32_t e = b - s > span ? s + span : b;
        quad_range<U, BF>(oadj4, seg, NZ, s, e, add);
        flush();
        s = e;
    }
}

// One chunk of up to TS middles (j = this thread's middle, valid below m1):
// reads each middle's descriptor, takes its segment, and compacts the
// non-empty segments into sm.seg with their prefix in quads (QUADS) or in
// wedges. T = the chunk's quads or wedges, NZ = its segments (the same in
// every thread of the team).
template <int TS, bool QUADS = true, typename Seg>
__device__ __forceinline__ void chunk_scan(const uint4 *__restrict__ smd, int64_t rb, uint32_t j,
                                           uint32_t m1, WalkSmem<TS> &sm, int t, Seg &&seg,
                                           uint32_t &T, uint32_t &NZ) {
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

// Walk the wedges of one anchor's middles [m0, m1) (its row starts at rb in
// the anchor side's descriptors smd; the middles' rows are in oadj) as a
// team of TS threads (t = thread index in the team): per chunk of TS
// middles, a chunk scan and then each thread's equal share of the chunk's
// quads. seg(md, st, len) picks the segment [st, st+len) of a middle's row
// from its descriptor; add is called as in quad_range, once per wedge
// (entry = endpoint side rank << 1 | sign of the middle-endpoint edge).
// flush() follows every `span` quads of a thread.
template <int TS, int U, bool BF, typename Seg, typename Add, typename Flush>
__device__ __forceinline__ void quad_walk(const uint4 *__restrict__ smd,
                                          const uint32_t *__restrict__ oadj, int64_t rb,
                                          uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                          uint32_t span, Seg &&seg, Add &&add, Flush &&flush) {
    const uint4 *oadj4 = reinterpret_cast<const uint4 *>(oadj);
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ;
        chunk_scan<TS>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ);
        quad_range_flushed<U, BF>(oadj4, sm.seg, NZ, share<TS>(T, t), share<TS>(T, t + 1), span,
                                  add, flush);
        team_sync<TS>();
    }
}

// Team walker in coalesced rounds. After the chunk scan each warp of the
// team takes an equal part [A, B) of the chunk's quads and walks it in
// rounds of 32 consecutive quads, lane l taking quad r + l (a round reads
// up to 512 consecutive bytes of a segment). The segments that start inside
// a round are found from the next 32 compacted segments, one per lane, whose
// starts form a bitmask (one warp OR-reduction); a lane's segment is the
// last one starting at or before its quad. Each round's quads are loaded one
// round ahead. add is called as in quad_range (BF chooses the form);
// flush() follows every `span` rounds of a warp and the end of its part.
template <int TS, bool BF, typename Seg, typename Add, typename Flush>
__device__ __forceinline__ void team_rounds(const uint4 *__restrict__ smd,
                                            const uint32_t *__restrict__ oadj, int64_t rb,
                                            uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                            uint32_t span, Seg &&seg, Add &&add, Flush &&flush) {
    constexpr uint32_t NW = TS / 32;
    const uint4 *oadj4 = reinterpret_cast<const uint4 *>(oadj);
    const uint32_t lane = (uint32_t)t & 31u, w = (uint32_t)t >> 5;
    const unsigned upto = (2u << lane) - 1u;
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ;
        chunk_scan<TS>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ);
        const uint32_t A = share<NW>(T, w), B = share<NW>(T, w + 1);
        if (A < B) {
            uint32_t kb = 0, hi = NZ;  // segment holding quad A
            while (kb < hi) {
                const uint32_t mid = (kb + hi) >> 1;
                if (sm.seg[mid].incl <= A) kb = mid + 1; else hi = mid;
            }
            kb++;  // next segment to start
            // lane's quad of the round at r: loads it, sets vm (0 past B) and sw
            auto locate = [&](uint32_t r, uint4 &v, uint32_t &vm, uint32_t &swq) {
                const uint32_t c = kb + lane;
                const uint32_t s = c < NZ ? (sm.seg[c].excl_sw & EXMASK) - r : 32u;
                const unsigned M = __reduce_or_sync(FULL, s < 32u ? 1u << s : 0u);
                const uint32_t k = kb - 1u + __popc(M & upto);
                kb += __popc(M);
                const uint32_t q = r + lane;
                vm = 0u;
                if (q < B) {
                    const QSeg d = sm.seg[k];
                    const uint32_t qq = (d.st >> 2) + (q - (d.excl_sw & EXMASK));
                    const uint32_t w0 = qq << 2;
                    const uint32_t lo = d.st > w0 ? d.st - w0 : 0u;
                    const uint32_t hq = d.en - w0 < 4u ? d.en - w0 : 4u;
                    vm = (0xfu >> (4u - hq)) & (0xfu << lo);
                    swq = d.excl_sw >> 31;
                    v = __ldg(oadj4 + qq);
                }
            };
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            uint32_t vm = 0u, swq = 0u, rounds = 0u;
            locate(A, v, vm, swq);
            for (uint32_t r = A; r < B; r += 32) {
                uint4 vn = make_uint4(0u, 0u, 0u, 0u);
                uint32_t vmn = 0u, swn = 0u;
                if (r + 32 < B) locate(r + 32, vn, vmn, swn);
                if constexpr (BF) {
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
                if (++rounds == span) { flush(); rounds = 0u; }
            }
            flush();
        }
        team_sync<TS>();
    }
}

// ------------------------------------------- bulk-copy staging (async proxy)
// Shared-memory mbarriers and non-multicast bulk copies from this GPU's
// global memory into the CTA's own shared memory (PTX cp.async.bulk with
// mbarrier::complete_tx).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bytes (a multiple of 16, 16-byte aligned source and destination)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bounded wait for phase `parity` of an mbarrier: false after MBAR_SPINS
// tries (try_wait itself blocks for a short time per try), so a copy that
// never lands turns into an error status instead of a hang.
constexpr uint32_t MBAR_SPINS = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < MBAR_SPINS; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Per warp: S stages of one round (32 quads) each, each lane's entry mask
// and sign for its quad of the stage, and the stages' mbarriers.
template <int S>
struct alignas(16) StageRing {
    uint4 q[S][32];
    uint32_t meta[S][32];
    unsigned long long bar[S];
};

// team_rounds with the adjacency staged in shared memory by bulk copies:
// the round at r is copied S - 1 rounds ahead of its use. Per round, the
// lane at the head of each run of lanes in one segment copies that run's
// quads (contiguous in the middle's row, 16-byte aligned) into the stage in
// one cp.async.bulk; lane 0 arms the stage's mbarrier with the round's
// bytes. A lane then reads its quad from the stage. `ring` is this warp's
// ring; its mbarriers are initialised once per kernel (stage_ring_init).
template <int S>
__device__ __forceinline__ void stage_ring_init(StageRing<S> &ring, unsigned lane) {
    if (lane == 0) {
        for (int k = 0; k < S; k++) mbar_init(smem_addr(&ring.bar[k]), 1);
        fence_mbar_init();
    }
    __syncwarp();
}

// Per-warp state of the staged walker across jobs: the parity of each
// stage's next phase, and whether the warp may still copy (a wait that gave
// up turns it off for the rest of the kernel: its copies are drained, its
// later rounds skipped, the error word set).
struct StageState {
    uint32_t phase = 0;
    bool ok = true;
};

template <int TS, int S, typename Seg, typename Add, typename Flush>
__device__ __forceinline__ void team_rounds_bulk(const uint4 *__restrict__ smd,
                                                 const uint32_t *__restrict__ oadj, int64_t rb,
                                                 uint32_t m0, uint32_t m1, WalkSmem<TS> &sm,
                                                 StageRing<S> &ring, StageState &ss, int t,
                                                 uint32_t span, uint32_t *err, Seg &&seg,
                                                 Add &&add, Flush &&flush) {
    constexpr uint32_t NW = TS / 32;
    const uint4 *oadj4 = reinterpret_cast<const uint4 *>(oadj);
    const uint32_t lane = (uint32_t)t & 31u, w = (uint32_t)t >> 5;
    const unsigned upto = (2u << lane) - 1u;
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ;
        chunk_scan<TS>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ);
        const uint32_t A = share<NW>(T, w), B = share<NW>(T, w + 1);
        if (A < B && ss.ok) {
            uint32_t kb = 0, hi = NZ;  // segment holding quad A
            while (kb < hi) {
                const uint32_t mid = (kb + hi) >> 1;
                if (sm.seg[mid].incl <= A) kb = mid + 1; else hi = mid;
            }
            kb++;
            const uint32_t nrounds = (B - A + 31) / 32;
            // issues round j (quads A + 32 j ..) into stage j % S
            auto issue = [&](uint32_t j) {
                const uint32_t r = A + 32 * j, st = j % S;
                const uint32_t c = kb + lane;
                const uint32_t s0 = c < NZ ? (sm.seg[c].excl_sw & EXMASK) - r : 32u;
                const unsigned M = __reduce_or_sync(FULL, s0 < 32u ? 1u << s0 : 0u);
                const uint32_t k = kb - 1u + __popc(M & upto);
                kb += __popc(M);
                const uint32_t q = r + lane;
                const uint32_t nv = B - r < 32u ? B - r : 32u;  // valid lanes this round
                uint32_t vm = 0u, swq = 0u, qq = 0u;
                if (q < B) {
                    const QSeg d = sm.seg[k];
                    qq = (d.st >> 2) + (q - (d.excl_sw & EXMASK));
                    const uint32_t w0 = qq << 2;
                    const uint32_t lo = d.st > w0 ? d.st - w0 : 0u;
                    const uint32_t hq = d.en - w0 < 4u ? d.en - w0 : 4u;
                    vm = (0xfu >> (4u - hq)) & (0xfu << lo);
                    swq = d.excl_sw >> 31;
                }
                ring.meta[st][lane] = vm | swq << 4;
                const uint32_t bar = smem_addr(&ring.bar[st]);
                fence_proxy_async();  // this stage's last reads before the new copy
                if (lane == 0) mbar_arrive_expect_tx(bar, nv * 16u);
                __syncwarp();
                // a run starts at lane 0 and at every segment start in the round
                const unsigned heads = (M | 1u) & ((nv == 32u) ? FULL : ((1u << nv) - 1u));
                if (q < B && ((heads >> lane) & 1u)) {
                    const unsigned later = heads & ~upto;  // heads after this lane
                    const uint32_t end = later ? (uint32_t)(__ffs(later) - 1) : nv;
                    bulk_g2s(smem_addr(&ring.q[st][lane]), oadj4 + qq, (end - lane) * 16u, bar);
                }
            };
            uint32_t issued = nrounds < (uint32_t)(S - 1) ? nrounds : (uint32_t)(S - 1);
            for (uint32_t j = 0; j < issued; j++) issue(j);
            uint32_t rounds = 0u;
            for (uint32_t j = 0; j < nrounds; j++) {
                if (issued < nrounds) issue(issued++);
                const uint32_t st = j % S;
                // all lanes take the same branch (one lane's wait may give up
                // while another's sees the phase complete)
                const bool landed = mbar_wait(smem_addr(&ring.bar[st]), (ss.phase >> st) & 1u);
                if (!__all_sync(FULL, landed)) {
                    // give up: drain every copy issued and not yet consumed
                    // (again bounded), then stop copying for good
                    set_error(err, E_WAIT);
                    for (uint32_t i = j; i < issued; i++)
                        mbar_wait(smem_addr(&ring.bar[i % S]), (ss.phase >> (i % S)) & 1u);
                    ss.ok = false;
                    break;
                }
                ss.phase ^= 1u << st;
                const uint32_t meta = ring.meta[st][lane];
                const uint32_t vm = meta & 0xfu, swq = meta >> 4;
                if (vm) {
                    const uint4 v = ring.q[st][lane];
                    add(v.x, vm & 1u, swq);
                    add(v.y, (vm >> 1) & 1u, swq);
                    add(v.z, (vm >> 2) & 1u, swq);
                    add(v.w, vm >> 3, swq);
                }
                __syncwarp();
                if (++rounds == span) { flush(); rounds = 0u; }
            }
            flush();
        }
        team_sync<TS>();
    }
}

// Wedge walker, per thread: the wedges [a, b) of a compacted chunk whose
// prefix is in wedges, U loads in flight per step, one(entry, sign bit of
// the anchor's edge) per wedge. For segment families whose per-wedge work
// is a loop (hash probes): one call site, no predicated quad entries.
template <int U, typename One>
__device__ __forceinline__ void wedge_range(const uint32_t *__restrict__ oadj, const QSeg *seg,
                                            uint32_t NZ, uint32_t a, uint32_t b, One &&one) {
    if (a >= b) return;
    uint32_t k = 0, hi = NZ;  // segment holding wedge a
    while (k < hi) {
        const uint32_t mid = (k + hi) >> 1;
        if (seg[mid].incl <= a) k = mid + 1; else hi = mid;
    }
    QSeg d = seg[k];
    uint32_t p = d.st + (a - (d.excl_sw & EXMASK));
    for (uint32_t i = a; i < b; i += U) {
        uint32_t pa[U], sq[U];
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
        }
        uint32_t xv[U];
#pragma unroll
        for (int u = 0; u < U; u++) xv[u] = pa[u] != 0xffffffffu ? __ldg(oadj + pa[u]) : 0u;
        for (int u = 0; u < U; u++)
            if (pa[u] != 0xffffffffu) one(xv[u], sq[u]);
    }
}

// quad_walk's counterpart over wedges (wedge_range per thread)
template <int TS, int U, typename Seg, typename One, typename Flush>
__device__ __forceinline__ void wedge_walk(const uint4 *__restrict__ smd,
                                           const uint32_t *__restrict__ oadj, int64_t rb,
                                           uint32_t m0, uint32_t m1, WalkSmem<TS> &sm, int t,
                                           uint32_t span, Seg &&seg, One &&one, Flush &&flush) {
    for (uint32_t mc = m0; mc < m1; mc += TS) {
        uint32_t T, NZ;
        chunk_scan<TS, false>(smd, rb, mc + (uint32_t)t, m1, sm, t, seg, T, NZ);
        const uint32_t a = share<TS>(T, t), b = share<TS>(T, t + 1);
        for (uint32_t s0 = a; s0 < b;) {
            const uint32_t e = b - s0 > span ? s0 + span : b;
            wedge_range<U>(oadj, sm.seg, NZ, s0, e, one);
            flush();
            s0 = e;
        }
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
// oneb(x, sw) one wedge of the second family; sw is the sign bit of the
// anchor's edge to the middle.
template <typename SegA, typename QuadA, typename SegB, typename OneB>
__device__ __forceinline__ void warp_rounds(const uint4 *__restrict__ smd,
                                            const uint32_t *__restrict__ oadj, int64_t rb,
                                            uint32_t m0, uint32_t m1, WalkSmem<32> &sa,
                                            WalkSmem<32> &sb, unsigned lane, SegA &&sega,
                                            QuadA &&quada, SegB &&segb, OneB &&oneb) {
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
        if (qa > 0)
            sa.seg[__popc(nza & upto) - 1] =
                QSeg{(uint32_t)sta, (uint32_t)sta + la, ea | (sw << 31), xa};
        if (lb > 0)
            sb.seg[__popc(nzb & upto) - 1] =
                QSeg{(uint32_t)stb, (uint32_t)stb + lb, eb | (sw << 31), xb};
        const uint32_t TA = __shfl_sync(FULL, xa, 31), TB = __shfl_sync(FULL, xb, 31);
        __syncwarp();
        // The second family's first round is loaded before the first
        // family's rounds run, and each round of the first family loads its
        // quads one round ahead: a warp keeps two loads in flight instead of
        // waiting out one memory round trip per round.
        uint32_t xb0 = 0, swb0 = 0, baseb = 0;
        bool hb0 = false;
        if (TB > 0) {
            const unsigned M = __reduce_or_sync(FULL, (lb > 0 && eb < 32u) ? 1u << eb : 0u);
            const uint32_t k = __popc(M & upto) - 1u;
            baseb = __popc(M);
            if (lane < TB) {
                const QSeg d = sb.seg[k];
                xb0 = oadj[d.st + (lane - (d.excl_sw & EXMASK))];
                swb0 = d.excl_sw >> 31;
                hb0 = true;
            }
        }
        uint32_t base = 0;  // segments of the first family starting before the next round
        // quad of lane `lane` in the round starting at quad r: loads it and
        // sets vm (0 past the chunk's quads) and sw
        auto locate = [&](uint32_t r, uint4 &v, uint32_t &vm, uint32_t &swq) {
            const uint32_t s = ea - r;
            const unsigned M = __reduce_or_sync(FULL, (qa > 0 && s < 32u) ? 1u << s : 0u);
            const uint32_t k = base + __popc(M & upto) - 1u;
            base += __popc(M);
            const uint32_t q = r + lane;
            vm = 0u;
            if (q < TA) {
                const QSeg d = sa.seg[k];
                const uint32_t qq = (d.st >> 2) + (q - (d.excl_sw & EXMASK));
                const uint32_t w0 = qq << 2;
                const uint32_t lo = d.st > w0 ? d.st - w0 : 0u;
                const uint32_t hi = d.en - w0 < 4u ? d.en - w0 : 4u;
                vm = (0xfu >> (4u - hi)) & (0xfu << lo);
                swq = d.excl_sw >> 31;
                v = __ldg(oadj4 + qq);
            }
        };
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        uint32_t vm = 0u, swq = 0u;
        if (TA > 0) locate(0, v, vm, swq);
        for (uint32_t r = 0; r < TA; r += 32) {
            uint4 vn = make_uint4(0u, 0u, 0u, 0u);
            uint32_t vmn = 0u, swn = 0u;
            if (r + 32 < TA) locate(r + 32, vn, vmn, swn);
            if (vm) quada(v, vm, swq);
            v = vn;
            vm = vmn;
            swq = swn;
        }
        if (hb0) oneb(xb0, swb0);
        for (uint32_t r = 32; r < TB; r += 32) {
            const uint32_t s = eb - r;
            const unsigned M = __reduce_or_sync(FULL, (lb > 0 && s < 32u) ? 1u << s : 0u);
            const uint32_t k = baseb + __popc(M & upto) - 1u;
            baseb += __popc(M);
            const uint32_t p = r + lane;
            if (p < TB) {
                const QSeg d = sb.seg[k];
                oneb(oadj[d.st + (p - (d.excl_sw & EXMASK))], d.excl_sw >> 31);
            }
        }
        __syncwarp();
    }
}

// Open-addressing tables in shared memory of 2^(32-shift) u64 slots: the
// key (endpoint + 1; 0 = empty) in the high half and the packed tallies
// (S | A << 16) in the low half. hash_add inserts or finds the key and adds
// inc to its tallies (an insert sets key and first tally in one
// compare-and-swap); it returns the tallies the key held before.
__device__ __forceinline__ uint32_t hash_add(unsigned long long *tab, uint32_t shift,
                                             uint32_t mask, uint32_t key, uint32_t inc,
                                             uint32_t *err) {
    uint32_t h = hash_slot(key, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const unsigned long long cur = *((volatile unsigned long long *)&tab[h]);
        const uint32_t k = (uint32_t)(cur >> 32);
        if (k == key) return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
        if (k == 0) {
            const unsigned long long want = ((unsigned long long)key << 32) | inc;
            const unsigned long long old = atomicCAS(&tab[h], 0ull, want);
            if (old == 0ull) return 0u;
            if ((uint32_t)(old >> 32) == key)
                return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
        }
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
__device__ __forceinline__ void hash_wedge32(unsigned long long *tab, uint32_t shift,
                                             uint32_t mask, uint32_t x, uint32_t sw,
                                             uint32_t *err, uint32_t &own, uint32_t &other) {
    const uint32_t asym = (x ^ sw) & 1u;
    const uint32_t old = hash_add(tab, shift, mask, (x >> 1) + 1, asym ? INC_ASYM : INC_SYM, err);
    const uint32_t pick = 1u << (asym << 3);
    own = __dp2a_lo(old, pick, own);
    other = __dp2a_lo(old, pick ^ 0x0101u, other);
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

// one warp-class anchor, walked by one warp
__device__ __forceinline__ void warp_anchor(const DevGraph &G, WarpSmem &sm, const AnchorRec &rec,
                                            unsigned lane, unsigned long long &bal,
                                            unsigned long long &tot) {
    uint32_t *err = &G.scratch->err;
    const Anchor A = load_anchor(G, rec);
    const uint64_t W = A.W, above = (uint64_t)(A.ns - A.r - 1);
    uint32_t cap = 0, shift = 0;
    // 32-bit sums: an anchor has at most WARP_W_MAX wedges, each adding less
    // than 2^8 to each sum (tallies are bounded by the degree <= WARP_DEG_MAX)
    static_assert(WARP_W_MAX * WARP_DEG_MAX < (1ull << 32), "32-bit warp sums");
    uint32_t own = 0, other = 0;
    auto none = [](const uint4 &, long long &st, uint32_t &len) { st = 0; len = 0; };
    auto no_quad = [](const uint4 &, uint32_t, uint32_t) {};
    if (rec.flags & REC_HASH_ALL) {  // hash every endpoint
        table_geometry(W < above ? W : above, 32, WARP_CAP, cap, shift);
        const uint32_t mask = cap - 1;
        warp_rounds(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, sm.walk2, lane, none, no_quad,
                    FullSeg{}, [&](uint32_t x, uint32_t sw) {
                        hash_wedge32(sm.tab, shift, mask, x, sw, err, own, other);
                    });
    } else {
        const int64_t ns = A.ns;
        const uint32_t wb = ns > (int64_t)HUB_WINDOW ? (uint32_t)(ns - HUB_WINDOW) : 0u;
        const uint64_t wnh = A.wnh;
        const uint64_t above_nh = wb > A.r + 1 ? (uint64_t)wb - A.r - 1 : 0;
        if (wnh > 0) table_geometry(wnh < above_nh ? wnh : above_nh, 32, WARP_CAP, cap, shift);
        const uint32_t mask = cap - 1;
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
                    LowSeg{}, [&](uint32_t x, uint32_t sw) {
                        hash_wedge32(sm.tab, shift, mask, x, sw, err, own, other);
                    });
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = lane; q < HUB_WINDOW / 8; q += 32) w4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    bal += own;
    tot += (unsigned long long)own + other;
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

__global__ void __launch_bounds__(WARP_THREADS, 4) k_warp(DevGraph G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned lane = lane_id();
    WarpSmem &sm = warp_smem_init(smem_raw, lane);
    const uint32_t n = G.ctr[CTR_WARP];
    const uint32_t gw = (blockIdx.x * WARP_THREADS + threadIdx.x) >> 5;
    const uint32_t GW = (gridDim.x * WARP_THREADS) >> 5;
    unsigned long long bal = 0, tot = 0;
    // the next anchor's record is loaded while this one is walked
    AnchorRec cur;
    if (gw < n) cur = G.warp_list[gw];
    for (uint32_t idx = gw; idx < n; idx += GW) {
        AnchorRec nxt;
        if (idx + GW < n) nxt = G.warp_list[idx + GW];
        warp_anchor(G, sm, cur, lane, bal, tot);
        spill_if_large(G.scratch, bal, tot);
        cur = nxt;
    }
    flush_warp(G.scratch, bal, tot);
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
    // hub walk: hb = the wedges' own previous tallies, ht = both previous
    // tallies; hash walk: own and other as in hash_wedge32
    // quads per thread step (per-thread quad shares measured faster than
    // warp rounds for these classes)
    constexpr int QU = TS == TEAM_THREADS ? 1 : 2;
    uint32_t hb = 0, ht = 0, own = 0, other = 0;
    auto flush = [&]() {
        bal += (unsigned long long)hb + own;
        tot += (unsigned long long)ht + own + other;
        hb = ht = own = other = 0;
    };
    if (W > wnh) {  // endpoints inside the hub window
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
    uint32_t cap = 0;
    if (wnh > 0) {  // endpoints below the window
        uint32_t shift;
        table_geometry(wnh < above_nh ? wnh : above_nh, 32, HCAP, cap, shift);
        const uint32_t mask = cap - 1;
        wedge_walk<TS, 2>(A.smd, A.oadj, A.rb, 0, A.deg, sm.walk, t, 4 * SUM_SPAN, LowSeg{},
                          [&](uint32_t x, uint32_t sw) {
                              hash_wedge32(sm.tab, shift, mask, x, sw, err, own, other);
                          },
                          flush);
    }
    __syncthreads();
    if (W > wnh) {
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = t; q < HUB_WINDOW / 4; q += TS) w4[q] = make_uint4(0u, 0u, 0u, 0u);
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
// Two dense walkers (a launch choice): STAGED CTAs stage the middles' rows
// in shared memory by bulk copies (DENSE_STAGES rounds per warp in flight;
// the rings cost a CTA per SM); otherwise each lane loads its quads itself,
// one round ahead. On the 2M x 500k graph the direct loads measured faster
// (1.63 against 2.58 ms) and are the default.
constexpr int DENSE_STAGES = 4;

template <bool STAGED>
struct alignas(16) DenseSmem {
    uint32_t cnt[DENSE_CAP];
    WalkSmem<DENSE_THREADS> walk;
    StageRing<DENSE_STAGES> ring[STAGED ? DENSE_THREADS / 32 : 1];
    uint32_t job, last;
};

// one dense job (an anchor, or one middle slice of a split anchor), walked
// by the whole CTA; adds each thread's part of its sums to bal and tot
template <bool STAGED>
__device__ __forceinline__ void dense_job(const DevGraph &G, DenseSmem<STAGED> &sm,
                                          const DenseJob &J, StageState &ss,
                                          unsigned long long &bal, unsigned long long &tot) {
    const int t = threadIdx.x;
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
        // b32: the wedges' own previous tallies; t32: both previous tallies.
        // The segments hold only endpoints in [e0, e1): the mask keeps a
        // counter index inside the array whatever the entry; an entry
        // outside its segment (vb = 0) adds 0 and picks nothing.
        uint32_t b32 = 0, t32 = 0;
        auto add = [&](uint32_t x, uint32_t vb, uint32_t sw) {
            const uint32_t asym = (x ^ sw) & 1u;
            const uint32_t idx = ((x >> 1) - e0) & (DENSE_CAP - 1);
            const uint32_t old = atomicAdd(&sm.cnt[idx], vb << (asym << 4));
            b32 = __dp2a_lo(old, vb << (asym << 3), b32);
            t32 = __dp2a_lo(old, vb * 0x0101u, t32);
        };
        auto flush = [&]() {
            bal += b32;
            tot += t32;
            b32 = t32 = 0;
        };
        auto clipped = [&](const uint4 &d, long long &st, uint32_t &l) {
            const long long s0 = lower_bound_u32(A.oadj, d.x, d.z, e0 << 1);
            st = s0;
            l = (uint32_t)(lower_bound_u32(A.oadj, s0, d.z, e1 << 1) - s0);
        };
        if constexpr (STAGED) {
            StageRing<DENSE_STAGES> &ring = sm.ring[t >> 5];
            if (windows)
                team_rounds_bulk<DENSE_THREADS, DENSE_STAGES>(A.smd, A.oadj, A.rb, J.m0, J.m1,
                                                              sm.walk, ring, ss, t, SUM_SPAN,
                                                              &G.scratch->err, clipped, add, flush);
            else
                team_rounds_bulk<DENSE_THREADS, DENSE_STAGES>(A.smd, A.oadj, A.rb, J.m0, J.m1,
                                                              sm.walk, ring, ss, t, SUM_SPAN,
                                                              &G.scratch->err, FullSeg{}, add,
                                                              flush);
        } else {
            if (windows)
                team_rounds<DENSE_THREADS, true>(A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t,
                                                 SUM_SPAN, clipped, add, flush);
            else
                team_rounds<DENSE_THREADS, true>(A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t,
                                                 SUM_SPAN, FullSeg{}, add, flush);
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

// One wide job (group WIDE_JOB): an anchor of degree above MAX_DEGREE,
// walked whole by the CTA with 64-bit counters, S in the low and A in the
// high half (each at most the degree < 2^32), over windows of DENSE_CAP / 2
// endpoints in the same shared memory. Each wedge adds the previous values
// of its own tally (balanced) and of both tallies (total) to 64-bit sums,
// which go to the grid accumulator before they could reach 2^53.
template <bool STAGED>
__device__ __forceinline__ void dense_job_wide(const DevGraph &G, DenseSmem<STAGED> &sm,
                                               const DenseJob &J, unsigned long long &bal,
                                               unsigned long long &tot) {
    constexpr uint32_t CAP = DENSE_CAP / 2;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(sm.cnt);
    const int t = threadIdx.x;
    const SideCSR &S = (J.anchor & 1u) ? G.side[1] : G.side[0];
    AnchorRec rec;
    rec.anchor = J.anchor;
    rec.rb = (uint32_t)S.off[J.anchor >> 1];
    rec.deg = 0; rec.W = 0; rec.wnh = 0;
    const Anchor A = load_anchor(G, rec);
    const uint32_t e_lo = A.r + 1, e_hi = (uint32_t)A.ns;
    const bool windows = (e_hi - e_lo) > CAP;
    for (uint32_t e0 = e_lo; e0 < e_hi; e0 += CAP) {
        const uint32_t e1 = e_hi - e0 > CAP ? e0 + CAP : e_hi;
        for (uint32_t i = t; i < e1 - e0; i += DENSE_THREADS) cnt[i] = 0ull;
        __syncthreads();
        auto add = [&](uint32_t x, uint32_t vb, uint32_t sw) {
            const uint32_t asym = (x ^ sw) & 1u;
            const uint32_t idx = ((x >> 1) - e0) & (CAP - 1);
            const unsigned long long old =
                atomicAdd(&cnt[idx], (unsigned long long)vb << (asym << 5));
            const unsigned long long oS = old & 0xffffffffull, oA = old >> 32;
            if (vb) {
                bal += asym ? oA : oS;
                tot += oS + oA;
            }
        };
        auto flush = [&]() { spill_if_large(G.scratch, bal, tot); };
        if (windows) {
            team_rounds<DENSE_THREADS, true>(
                A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t, 1024,
                [&](const uint4 &d, long long &st, uint32_t &l) {
                    const long long s0 = lower_bound_u32(A.oadj, d.x, d.z, e0 << 1);
                    st = s0;
                    l = (uint32_t)(lower_bound_u32(A.oadj, s0, d.z, e1 << 1) - s0);
                },
                add, flush);
        } else {
            team_rounds<DENSE_THREADS, true>(A.smd, A.oadj, A.rb, J.m0, J.m1, sm.walk, t, 1024,
                                             FullSeg{}, add, flush);
        }
        __syncthreads();  // the next window rewrites the counters
    }
}

template <bool STAGED>
__global__ void __launch_bounds__(DENSE_THREADS, STAGED ? 2 : 3) k_dense(DevGraph G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DenseSmem<STAGED> &sm = *reinterpret_cast<DenseSmem<STAGED> *>(smem_raw);
    const uint32_t njobs = G.ctr[CTR_DENSE];
    StageState ss;
    if constexpr (STAGED) stage_ring_init(sm.ring[threadIdx.x >> 5], lane_id());
    unsigned long long bal = 0, tot = 0;  // summed over all jobs of this CTA
    for (;;) {
        if (threadIdx.x == 0) sm.job = atomicAdd(&G.scratch->job_next[CLS_DENSE], 1u);
        __syncthreads();
        const uint32_t jid = sm.job;
        __syncthreads();
        if (jid >= njobs) break;
        const DenseJob J = G.dense_jobs[jid];
        if (J.group != WIDE_JOB) dense_job(G, sm, J, ss, bal, tot);  // wide jobs: k_wide
        spill_if_large(G.scratch, bal, tot);
    }
    flush_warp(G.scratch, bal, tot);
}

// The wide jobs among the dense jobs (anchors of degree above MAX_DEGREE),
// one CTA per job; a kernel of their own keeps their 64-bit walk out of
// k_dense's registers. Exits at once when the graph has none.
__global__ void __launch_bounds__(DENSE_THREADS) k_wide(DevGraph G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DenseSmem<false> &sm = *reinterpret_cast<DenseSmem<false> *>(smem_raw);
    const uint32_t njobs = G.ctr[CTR_DENSE];
    unsigned long long bal = 0, tot = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t j = atomicAdd(&G.scratch->job_next[JOB_WIDE], 1u);
            while (j < njobs && G.dense_jobs[j].group != WIDE_JOB)
                j = atomicAdd(&G.scratch->job_next[JOB_WIDE], 1u);
            sm.job = j;
        }
        __syncthreads();
        const uint32_t jid = sm.job;
        __syncthreads();
        if (jid >= njobs) break;
        dense_job_wide(G, sm, G.dense_jobs[jid], bal, tot);
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
            warp_anchor(G, sm, G.warp_list[it - gbeg], lane, bal, tot);
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

template <bool STAGED>
__global__ void __launch_bounds__(DENSE_THREADS) k_dense_batch(BatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DenseSmem<STAGED> &sm = *reinterpret_cast<DenseSmem<STAGED> *>(smem_raw);
    StageState ss;
    if constexpr (STAGED) stage_ring_init(sm.ring[threadIdx.x >> 5], lane_id());
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
        const DenseJob J = G.dense_jobs[it - p[gi]];
        if (J.group == WIDE_JOB) dense_job_wide(G, sm, J, bal, tot);
        else dense_job(G, sm, J, ss, bal, tot);
        spill_if_large(G.scratch, bal, tot);
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
        for (int k = 0; k < 7; k++) sc->job_next[k] = 0;
        sc->err = 0;
    }
}

// every member's class counters and class statistics (after a
// re-classification), NCTR and 3 * NCLS words per graph
__global__ void k_batch_classes(BatchArgs B, uint32_t *ctr, unsigned long long *stats) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n; i += gridDim.x * blockDim.x) {
        const DevGraph &G = B.graphs[i];
        for (int k = 0; k < NCTR; k++) ctr[(size_t)i * NCTR + k] = G.ctr[k];
        for (int k = 0; k < 3 * NCLS; k++) stats[(size_t)i * 3 * NCLS + k] = G.cls_stats[k];
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
constexpr size_t DENSE_SMEM = sizeof(DenseSmem<false>);
constexpr size_t DENSE_SMEM_STAGED = sizeof(DenseSmem<true>);


struct LaunchCfg {
    int warp_blocks = 0, team_blocks = 0, ctah_blocks = 0, dense_blocks[2] = {};
    int batch_blocks[NCLS] = {};
    int dense_batch_blocks[2] = {};  // direct-load and staged dense batch kernels
    int sms = 0;
};

template <typename K>
int blocks_for(K kernel, int threads, size_t smem, int sms) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem);
    return std::max(1, b) * sms;
}

// Grids and shared-memory opt-ins, once per device (any thread may count on
// any device; the first launch on a device sets its entry up).
constexpr int MAX_DEVICES = 64;
LaunchCfg g_cfg[MAX_DEVICES];
std::once_flag g_cfg_once[MAX_DEVICES];

const LaunchCfg &init_cfg() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        dev = 0;
    }
    std::call_once(g_cfg_once[dev], [dev]() {
        LaunchCfg &c = g_cfg[dev];
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, dev);
        const int sms = prop.multiProcessorCount;
        c.sms = sms;
        c.warp_blocks = blocks_for(k_warp, WARP_THREADS, WARP_SMEM, sms);
        c.team_blocks = blocks_for(k_team, TEAM_THREADS, TEAM_SMEM, sms);
        c.ctah_blocks = blocks_for(k_ctah, CTAH_THREADS, CTAH_SMEM, sms);
        c.dense_blocks[0] = blocks_for(k_dense<false>, DENSE_THREADS, DENSE_SMEM, sms);
        c.dense_blocks[1] = blocks_for(k_dense<true>, DENSE_THREADS, DENSE_SMEM_STAGED, sms);
        blocks_for(k_wide, DENSE_THREADS, DENSE_SMEM, sms);  // shared-memory opt-in
        c.batch_blocks[CLS_WARP] = blocks_for(k_warp_batch, WARP_THREADS, WARP_SMEM, sms);
        c.batch_blocks[CLS_TEAM] = blocks_for(k_team_batch, TEAM_THREADS, TEAM_SMEM, sms);
        c.batch_blocks[CLS_CTAH] = blocks_for(k_ctah_batch, CTAH_THREADS, CTAH_SMEM, sms);
        c.dense_batch_blocks[0] = blocks_for(k_dense_batch<false>, DENSE_THREADS, DENSE_SMEM, sms);
        c.dense_batch_blocks[1] =
            blocks_for(k_dense_batch<true>, DENSE_THREADS, DENSE_SMEM_STAGED, sms);
        c.batch_blocks[CLS_DENSE] = c.dense_batch_blocks[0];
    });
    return g_cfg[dev];
}

}  // namespace

void count_init() { init_cfg(); }

void launch_count(const DevGraph &g, cudaStream_t s, int64_t *per_vertex_dev, cudaEvent_t *ev) {
    (void)per_vertex_dev;
    const LaunchCfg &cfg = init_cfg();
    cudaMemsetAsync(g.scratch, 0, sizeof(CountScratch), s);
    if (ev) record_timing_event(ev[0], s);
    if (g.dense_staged)
        k_dense<true><<<cfg.dense_blocks[1], DENSE_THREADS, DENSE_SMEM_STAGED, s>>>(g);
    else
        k_dense<false><<<cfg.dense_blocks[0], DENSE_THREADS, DENSE_SMEM, s>>>(g);
    note_launch();
    // wide jobs exist only when some degree exceeds the 16-bit tally range
    if (g.h_maxdeg > MAX_DEGREE) { k_wide<<<cfg.sms, DENSE_THREADS, DENSE_SMEM, s>>>(g); note_launch(); }
    if (ev) record_timing_event(ev[1], s);
    k_ctah<<<cfg.ctah_blocks, CTAH_THREADS, CTAH_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[2], s);
    k_team<<<cfg.team_blocks, TEAM_THREADS, TEAM_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[3], s);
    k_warp<<<cfg.warp_blocks, WARP_THREADS, WARP_SMEM, s>>>(g); note_launch();
    if (ev) record_timing_event(ev[4], s);
}

int batch_max_blocks(int cls) { return init_cfg().batch_blocks[cls]; }

void launch_count_batch(const BatchLaunch &L, const BatchTune &T, cudaStream_t s,
                        const cudaStream_t *side, const cudaEvent_t *ev, const cudaEvent_t *tev) {
    const LaunchCfg &cfg = init_cfg();
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
        const int full = c == CLS_DENSE ? cfg.dense_batch_blocks[T.dense_staged ? 1 : 0]
                                        : cfg.batch_blocks[c];
        int blocks = std::max(1, (int)(full * T.grid_frac[c] + 0.5f));
        blocks = std::min(blocks, full);
        if (c == CLS_WARP) {
            const uint64_t warps = ((uint64_t)L.items[c] + B.warp_chunk - 1) / B.warp_chunk;
            blocks = (int)std::min<uint64_t>(blocks, (warps + WARP_THREADS / 32 - 1) / (WARP_THREADS / 32));
            k_warp_batch<<<blocks, WARP_THREADS, WARP_SMEM, cs>>>(B);
        } else {
            blocks = (int)std::min<uint64_t>(blocks, L.items[c]);
            if (c == CLS_TEAM) k_team_batch<<<blocks, TEAM_THREADS, TEAM_SMEM, cs>>>(B);
            else if (c == CLS_CTAH) k_ctah_batch<<<blocks, CTAH_THREADS, CTAH_SMEM, cs>>>(B);
            else if (T.dense_staged)
                k_dense_batch<true><<<blocks, DENSE_THREADS, DENSE_SMEM_STAGED, cs>>>(B);
            else
                k_dense_batch<false><<<blocks, DENSE_THREADS, DENSE_SMEM, cs>>>(B);
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

void launch_batch_classes(const BatchLaunch &L, uint32_t *ctr_dev, unsigned long long *stats_dev,
                          cudaStream_t s) {
    BatchArgs B;
    B.graphs = L.graphs;
    B.prefix = L.prefix;
    B.next = L.next;
    B.n = L.n;
    B.warp_chunk = 1;
    const uint32_t blocks = std::min<uint32_t>((L.n + 255) / 256, 1024);
    if (L.n) { k_batch_classes<<<blocks, 256, 0, s>>>(B, ctr_dev, stats_dev); note_launch(); }
}

void launch_flip(DevGraph &g, const int64_t *edge_idx_dev, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_flip<<<(unsigned)blocks, 256, 0, s>>>(g, edge_idx_dev, n); note_launch();
}

}  // namespace bb
