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
#include "walk.cuh"

namespace bb {

namespace {

using namespace walk;

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
// ------------------------------------------------------------ warp class
// one warp-class anchor, walked by one warp: tally, then reset the counters
__device__ __forceinline__ void warp_anchor(const DevGraph &G, WarpSmem &sm, const AnchorRec &rec,
                                            unsigned lane, unsigned long long &bal,
                                            unsigned long long &tot) {
    const Anchor A = load_anchor(G, rec);
    uint32_t own = 0, other = 0;
    const WarpTab tb = warp_tally<true>(G, sm, rec, A, lane, own, other);
    if (!(rec.flags & REC_HASH_ALL)) {
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = lane; q < HUB_WINDOW / 8; q += 32) w4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    bal += own;
    tot += (unsigned long long)own + other;
    clear_table<32>(sm.tab, tb.cap, (int)lane);
    __syncwarp();
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
// one team/CTA-hash anchor, walked by the whole CTA: tally, then reset
template <int TS, uint32_t HCAP>
__device__ __forceinline__ void hybrid_anchor(const DevGraph &G, HybSmem<TS, HCAP> &sm,
                                              const AnchorRec &rec, unsigned long long &bal,
                                              unsigned long long &tot) {
    const int t = threadIdx.x;
    const Anchor A = load_anchor(G, rec);
    const HybTab tb = hybrid_tally<TS, HCAP>(G, sm, A, bal, tot);
    __syncthreads();
    if (tb.hub) {
        uint4 *w4 = reinterpret_cast<uint4 *>(sm.win);
        for (uint32_t q = t; q < HUB_WINDOW / 4; q += TS) w4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    clear_table<TS>(sm.tab, tb.cap, t);
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

bool launch_count(const DevGraph &g, cudaStream_t s, cudaEvent_t *ev) {
    const LaunchCfg &cfg = init_cfg();
    cudaMemsetAsync(g.scratch, 0, sizeof(CountScratch), s);
    if (ev) record_timing_event(ev[0], s);
    if (g.product_only || (g.prod.side >= 0 && product_enabled())) {
        const bool ok = launch_product(g, s);
        // a graph built for the product path alone has no classes to fall
        // back on (a failed launch has marked its error word instead)
        if (ok || g.product_only) {
            if (ev)
                for (int k = 1; k <= 4; k++) record_timing_event(ev[k], s);
            return ok;
        }
    }
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
    return false;
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
