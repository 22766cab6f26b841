// flips.cu - the change in the balanced count when a set F of edges flips
// sign, without recounting the whole graph (the incremental re-count under
// sign flips that follows the paper's edge-level extension).
//
// Flipping F toggles the balance of exactly the butterflies that contain an
// odd number of its edges: a balanced one becomes unbalanced (-1) and vice
// versa (+1); the total is unchanged. Every butterfly B through a flipped
// edge e = (a, b) is found once from e: a second vertex c in N(b) \ {a} on
// a's side and a common neighbour d of a and c other than b. A butterfly
// with k flipped edges is found from each of them, so it adds its change
// with weight 3/k (k = 1 or 3; even k adds nothing) and the sum is 3 times
// the change. The walk reads the signs before the flips are applied.
//
// Cost: from e the walk visits every c in N(b) and intersects two rows
// (each element of the shorter binary-searched in the longer). The side of
// a is chosen per edge to minimise sum over c of deg(c); the host compares
// the estimate for the whole set with the graph's wedge count (a step here
// costs well over a wedge of the count) and recounts when that is cheaper:
// with many flips on a power-law graph the enumeration exceeds a recount.
#include <algorithm>

#include "graph.cuh"

namespace bb {

namespace {

constexpr int FD_THREADS = 256;

// one flipped edge: side ranks, its positions in both sides' adjacency, and
// the side whose rows are intersected (0: a in U, 1: a in V)
struct FlipRec {
    uint32_t ru, rv;
    uint32_t pu, pv;
    uint32_t side;
    uint32_t pad[3];
};

__device__ __forceinline__ bool flagged(const uint32_t *f, uint32_t p) {
    return (f[p >> 5] >> (p & 31u)) & 1u;
}

// locate each flipped edge, mark it in both sides' flag bitmaps, and
// estimate its enumeration cost both ways (sum of the degrees of the other
// endpoint's neighbours); one warp per edge
__global__ void k_flip_locate(DevGraph G, const int64_t *edges, int64_t n, FlipRec *rec,
                              uint32_t *flagU, uint32_t *flagV, unsigned long long *cost) {
    const SideCSR &U = G.side[0];
    const SideCSR &V = G.side[1];
    const unsigned lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t e = edges[i];
        int64_t lo = 0, hi = G.nU;  // last u with rowptr[u] <= e
        while (hi - lo > 1) {
            const int64_t m = (lo + hi) >> 1;
            if (G.rowptr[m] <= e) lo = m; else hi = m;
        }
        const uint32_t ru = U.sr_of_id[lo];
        const uint32_t rv = V.sr_of_id[G.col[e]];
        const int64_t pu = lower_bound_u32(U.adj, U.off[ru], U.off[ru + 1], rv << 1);
        const int64_t pv = lower_bound_u32(V.adj, V.off[rv], V.off[rv + 1], ru << 1);
        // a in U: c runs over N(v) (U vertices); a in V: c runs over N(u)
        unsigned long long hv = 0, hu = 0;
        for (int64_t q = V.off[rv] + lane; q < V.off[rv + 1]; q += 32) {
            const uint32_t c = V.adj[q] >> 1;
            hv += (unsigned long long)(U.off[c + 1] - U.off[c]);
        }
        for (int64_t q = U.off[ru] + lane; q < U.off[ru + 1]; q += 32) {
            const uint32_t c = U.adj[q] >> 1;
            hu += (unsigned long long)(V.off[c + 1] - V.off[c]);
        }
        hv = warp_sum_u64(hv);
        hu = warp_sum_u64(hu);
        if (lane == 0) {
            FlipRec r;
            r.ru = ru; r.rv = rv;
            r.pu = (uint32_t)pu; r.pv = (uint32_t)pv;
            r.side = hv <= hu ? 0u : 1u;
            r.pad[0] = r.pad[1] = r.pad[2] = 0;
            rec[i] = r;
            atomicOr(&flagU[pu >> 5], 1u << (pu & 31));
            atomicOr(&flagV[pv >> 5], 1u << (pv & 31));
            atomicAdd(cost, hv <= hu ? hv : hu);
        }
    }
}

// 3 x (change in the balanced count): one CTA per flipped edge; its warps
// take the vertices c, its lanes the elements of the shorter row of a and c
__global__ void __launch_bounds__(FD_THREADS) k_flip_delta(DevGraph G, const FlipRec *rec,
                                                           int64_t n, const uint32_t *flagU,
                                                           const uint32_t *flagV,
                                                           unsigned long long *acc) {
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5, nwarps = FD_THREADS / 32;
    unsigned long long up = 0, down = 0;  // weighted +1 and -1 changes
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const FlipRec r = rec[i];
        const bool aU = r.side == 0;
        const SideCSR &A = aU ? G.side[0] : G.side[1];  // side of a (rows intersected)
        const SideCSR &B = aU ? G.side[1] : G.side[0];  // side of b
        const uint32_t *fA = aU ? flagU : flagV, *fB = aU ? flagV : flagU;
        const uint32_t a = aU ? r.ru : r.rv, b = aU ? r.rv : r.ru;
        const uint32_t pa_b = aU ? r.pu : r.pv;        // entry of b in row a
        const uint32_t s_ab = A.adj[pa_b] & 1u;
        const int64_t a0 = A.off[a], a1 = A.off[a + 1];
        for (int64_t qc = B.off[b] + warp; qc < B.off[b + 1]; qc += nwarps) {
            const uint32_t xc = B.adj[qc];
            const uint32_t c = xc >> 1;
            if (c == a) continue;
            const uint32_t s_cb = xc & 1u, f_cb = flagged(fB, (uint32_t)qc);
            const int64_t c0 = A.off[c], c1 = A.off[c + 1];
            // walk the shorter row, search the longer
            const bool a_short = (a1 - a0) <= (c1 - c0);
            const int64_t s0 = a_short ? a0 : c0, s1 = a_short ? a1 : c1;
            const int64_t l0 = a_short ? c0 : a0, l1 = a_short ? c1 : a1;
            for (int64_t ps = s0 + lane; ps < s1; ps += 32) {
                const uint32_t xs = A.adj[ps];
                const uint32_t d = xs >> 1;
                if (d == b) continue;
                const int64_t pl = lower_bound_u32(A.adj, l0, l1, d << 1);
                if (pl >= l1 || (A.adj[pl] >> 1) != d) continue;
                const uint32_t xl = A.adj[pl];
                const int64_t pad = a_short ? ps : pl, pcd = a_short ? pl : ps;
                const uint32_t s_ad = (a_short ? xs : xl) & 1u, s_cd = (a_short ? xl : xs) & 1u;
                const uint32_t k = 1u + flagged(fA, (uint32_t)pad) + f_cb +
                                   flagged(fA, (uint32_t)pcd);
                if (!(k & 1u)) continue;
                const unsigned long long w = k == 1 ? 3ull : 1ull;
                // balanced before (even number of negative edges) -> loses one
                if (((s_ab ^ s_ad ^ s_cb ^ s_cd) & 1u) == 0) down += w; else up += w;
            }
        }
    }
    up = warp_sum_u64(up);
    down = warp_sum_u64(down);
    if (lane == 0) {
        if (up) atomicAdd(&acc[0], up);
        if (down) atomicAdd(&acc[1], down);
    }
}


}  // namespace

size_t flip_ws_bytes(int64_t nE, int64_t n) {
    const size_t words = (size_t)(nE / 32 + 1);
    return ((size_t)n * sizeof(FlipRec) + 255) / 256 * 256 + 2 * ((words * 4 + 255) / 256 * 256) + 256;
}

void launch_flip_estimate(const DevGraph &g, const int64_t *edges_dev, int64_t n, void *ws,
                          unsigned long long *cost_dev, cudaStream_t s) {
    const size_t words = (size_t)(g.nE / 32 + 1);
    char *p = (char *)ws;
    FlipRec *rec = (FlipRec *)p;
    p += ((size_t)n * sizeof(FlipRec) + 255) / 256 * 256;
    uint32_t *flagU = (uint32_t *)p;
    p += (words * 4 + 255) / 256 * 256;
    uint32_t *flagV = (uint32_t *)p;
    cudaMemsetAsync(flagU, 0, words * 4, s);
    cudaMemsetAsync(flagV, 0, words * 4, s);
    cudaMemsetAsync(cost_dev, 0, 8, s);
    const int64_t blocks = std::min<int64_t>((n * 32 + 255) / 256, 4096);
    if (n > 0) { k_flip_locate<<<(unsigned)blocks, 256, 0, s>>>(g, edges_dev, n, rec, flagU, flagV, cost_dev); note_launch(); }
}

void launch_flip_delta(const DevGraph &g, int64_t n, void *ws, unsigned long long *acc_dev,
                       cudaStream_t s) {
    const size_t words = (size_t)(g.nE / 32 + 1);
    char *p = (char *)ws;
    FlipRec *rec = (FlipRec *)p;
    p += ((size_t)n * sizeof(FlipRec) + 255) / 256 * 256;
    uint32_t *flagU = (uint32_t *)p;
    p += (words * 4 + 255) / 256 * 256;
    uint32_t *flagV = (uint32_t *)p;
    cudaMemsetAsync(acc_dev, 0, 16, s);
    if (n <= 0) return;
    const int64_t blocks = std::min<int64_t>(n, 65535);
    k_flip_delta<<<(unsigned)blocks, FD_THREADS, 0, s>>>(g, rec, n, flagU, flagV, acc_dev); note_launch();
}

}  // namespace bb
