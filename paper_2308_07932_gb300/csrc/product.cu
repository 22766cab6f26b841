// product.cu - the matrix-product path for graphs with a small dense side
// (the plan and its exactness argument are in graph.cuh).
//
// Per pair (w, u) of the pair side P, over the middles v of the other side
// O: S = #{v : sign(w,v) sign(v,u) = +1} and A = #{v : = -1} are the pair's
// symmetric and asymmetric wedge tallies (Defs. 5-6), and by Lemma 2 the
// pair lies in C(S,2) + C(A,2) balanced and C(S+A,2) butterflies in all.
// With X the signed adjacency (X[w][v] = sign(w,v), 0 for no edge),
// (X X^T)[w][u] = S - A and (|X| |X|^T)[w][u] = S + A. On the caller's
// stream:
//   fill          X and |X| (bf16; the sums do not depend on the order of
//                 rows or columns). A fully built graph fills from its
//                 sign-packed rows of P (rows and columns in side-rank
//                 order; these rows carry later sign flips); a graph built
//                 for this path alone fills from the input rows (ids).
//                 k_prod_fill_rows stages a window of a row in shared
//                 memory and writes it whole; k_prod_fill scatters the
//                 entries after a clear (input rows with P = V, or rows too
//                 long to stage);
//   wedge count   (a graph built for this path alone) the priority wedges
//                 the library reports, from one pass over |X|: for a vertex
//                 of degree d with k neighbours ranked above it (Def. 4)
//                 C(d,2) - C(d-k,2) wedges have it as the middle and a
//                 higher-ranked vertex as the top (k_prod_degrees, then
//                 k_prod_wsum);
//   two strided-batched GEMMs (cuBLAS, bf16 in, fp32 sums) form both
//                 products, each as a batch of partial products over
//                 slices of the middles (ProductPlan::split);
//   k_prod_pairs  adds each pair's partials (in integers) and sums
//                 C(S,2) + C(A,2) and C(S+A,2) over the pairs w < u into the
//                 128-bit accumulators of the wedge classes; it also sums the
//                 diagonal of |X| |X|^T, the number of distinct nonzero cells,
//                 which k_prod_check compares with the edge count: an edge
//                 listed twice writes one cell twice and leaves it short.
#include <cublas_v2.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "walk.cuh"

namespace bb {

namespace {

using walk::acc_add;
using walk::block_sum2;
using walk::spill_if_large;

constexpr uint16_t BF16_PLUS_ONE = 0x3F80u;
constexpr uint16_t BF16_MINUS_ONE = 0xBF80u;
constexpr uint32_t BF16_ABS_MASK2 = 0x7FFF7FFFu;  // clears the sign bits of two bf16
constexpr int PROD_THREADS = 256;
// Row fill through shared memory: the matrix rows are cut into windows of
// at most FILL_WIN columns (64 KiB of bf16), one CTA per (row, window), as
// many windows per row as keep the GPU busy; a row whose entries would be
// scanned more than FILL_MAX_WINDOWS times is scattered instead.
constexpr uint32_t FILL_WIN = 32768;
constexpr uint32_t FILL_MAX_WINDOWS = 8;
constexpr size_t FILL_SMEM = FILL_WIN * sizeof(uint16_t);

// The rows a fill reads: the input rows (rowptr, col, sign; pair side U)
// or a side's built rows (off, adj: entry = column << 1 | negative).
struct FillRows {
    const int64_t *rowptr;
    const int32_t *col;
    const int8_t *sign;
    const uint32_t *adj;  // non-null: built rows (rowptr = the side's offsets)
    int64_t n;            // rows
    __device__ __forceinline__ void entry(int64_t p, uint32_t &c, bool &neg) const {
        if (adj) {
            const uint32_t x = adj[p];
            c = x >> 1;
            neg = x & 1u;
        } else {
            c = (uint32_t)col[p];
            neg = sign[p] < 0;
        }
    }
};

// CTA (blockIdx.x, blockIdx.y) = (window, row r < ap; rows past n are
// zero): the row's entries inside the window's width columns go into a
// zeroed shared copy, which then goes out in 16-byte stores to X and, with
// the sign bits cleared, to |X|.
__global__ void __launch_bounds__(PROD_THREADS) k_prod_fill_rows(FillRows R, uint32_t ld,
                                                                  uint32_t width, size_t plane,
                                                                  uint16_t *x) {
    extern __shared__ uint4 win4[];
    uint16_t *win = reinterpret_cast<uint16_t *>(win4);
    const int64_t r = blockIdx.y;
    const uint32_t c0 = blockIdx.x * width;
    if (c0 >= ld) return;  // (uniform over the CTA)
    const uint32_t w = ld - c0 < width ? ld - c0 : width;  // a multiple of 64
    for (uint32_t i = threadIdx.x; i < w / 8; i += PROD_THREADS) win4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int64_t b = r < R.n ? R.rowptr[r] : 0, e = r < R.n ? R.rowptr[r + 1] : 0;
    int64_t p = b + threadIdx.x;
    for (; p + 3 * PROD_THREADS < e; p += 4 * PROD_THREADS) {  // four entries in flight
        uint32_t c[4];
        bool neg[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            R.entry(p + k * PROD_THREADS, c[k], neg[k]);
            c[k] -= c0;  // wraps for columns before c0
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (c[k] < w) win[c[k]] = neg[k] ? BF16_MINUS_ONE : BF16_PLUS_ONE;
    }
    for (; p < e; p += PROD_THREADS) {
        uint32_t c;
        bool neg;
        R.entry(p, c, neg);
        c -= c0;
        if (c < w) win[c] = neg ? BF16_MINUS_ONE : BF16_PLUS_ONE;
    }
    __syncthreads();
    uint4 *xr = reinterpret_cast<uint4 *>(x + (size_t)r * ld + c0);
    uint4 *ar = reinterpret_cast<uint4 *>(x + plane + (size_t)r * ld + c0);
    for (uint32_t i = threadIdx.x; i < w / 8; i += PROD_THREADS) {
        const uint4 q = win4[i];
        xr[i] = q;
        ar[i] = make_uint4(q.x & BF16_ABS_MASK2, q.y & BF16_ABS_MASK2, q.z & BF16_ABS_MASK2,
                           q.w & BF16_ABS_MASK2);
    }
}

// one CTA per row u of R (grid-stride) into a cleared X and |X|: X[u][c]
// for each entry (u, c), or X[c][u] when `transpose` (input rows, pair
// side V)
__global__ void __launch_bounds__(PROD_THREADS) k_prod_fill(FillRows R, bool transpose,
                                                             uint32_t ld, size_t plane,
                                                             uint16_t *x) {
    for (int64_t u = blockIdx.x; u < R.n; u += gridDim.x) {
        const int64_t b = R.rowptr[u], e = R.rowptr[u + 1];
        for (int64_t p = b + threadIdx.x; p < e; p += PROD_THREADS) {
            uint32_t c;
            bool neg;
            R.entry(p, c, neg);
            const size_t cell = transpose ? (size_t)c * ld + (size_t)u : (size_t)u * ld + c;
            x[cell] = neg ? BF16_MINUS_ONE : BF16_PLUS_ONE;
            x[plane + cell] = BF16_PLUS_ONE;
        }
    }
}

// global priority rank of every vertex by id: P's a, then O's b
__global__ void k_prod_gid(SideCSR P, SideCSR O, uint32_t a, uint32_t b, uint32_t *gid) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a + b; i += gridDim.x * blockDim.x)
        gid[i] = i < a ? P.grank[P.sr_of_id[i]] : O.grank[O.sr_of_id[i - a]];
}

// Per row p and column o of |X|: its cells (the degree) and the cells whose
// other vertex is ranked above it. A thread takes 8 consecutive columns of
// the rows [blockIdx.y * rows, ...) (rows <= DEG_ROWS): row figures are
// reduced per warp, then across the block's warps in shared memory, column
// figures per thread; each is then added to its counter once per block.
constexpr uint32_t DEG_ROWS = 128;
__global__ void __launch_bounds__(PROD_THREADS) k_prod_degrees(
    const uint16_t *__restrict__ ax, uint32_t a, uint32_t b, uint32_t ld, uint32_t rows,
    const uint32_t *__restrict__ gid, uint32_t *row_d, uint32_t *row_k, uint32_t *col_d,
    uint32_t *col_k) {
    const uint32_t c8 = blockIdx.x * PROD_THREADS + threadIdx.x;
    const bool live = c8 * 8u < ld;  // every lane takes part in the row reductions
    const uint32_t *go = gid + a;
    uint32_t gcol[8], dc[8], kc[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t c = c8 * 8u + j;
        gcol[j] = live && c < b ? go[c] : 0u;
        dc[j] = kc[j] = 0u;
    }
    __shared__ uint32_t s_d[DEG_ROWS][PROD_THREADS / 32], s_k[DEG_ROWS][PROD_THREADS / 32];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t p0 = blockIdx.y * rows, p1 = p0 + rows < a ? p0 + rows : a;
    constexpr uint32_t RU = 4;  // rows whose loads are in flight together
    for (uint32_t pb = p0; pb < p1; pb += RU) {
        uint4 q[RU];
        uint32_t gp[RU];
#pragma unroll
        for (uint32_t i = 0; i < RU; i++) {
            const uint32_t p = pb + i;
            q[i] = make_uint4(0u, 0u, 0u, 0u);
            gp[i] = p < p1 ? gid[p] : 0u;
            if (live && p < p1) q[i] = reinterpret_cast<const uint4 *>(ax + (size_t)p * ld)[c8];
        }
#pragma unroll
        for (uint32_t i = 0; i < RU; i++) {
            if (pb + i >= p1) break;  // (uniform over the block)
            const uint32_t w[4] = {q[i].x, q[i].y, q[i].z, q[i].w};
            uint32_t dr = 0, kr = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const uint32_t nz = ((w[j >> 1] >> ((j & 1) * 16)) & 0x7FFFu) != 0u;
                dc[j] += nz;
                kc[j] += nz & (gp[i] > gcol[j]);
                dr += nz;
                kr += nz & (gcol[j] > gp[i]);
            }
            dr = warp_sum_u32(dr);
            kr = warp_sum_u32(kr);
            if (lane_id() == 0) {
                s_d[pb + i - p0][warp] = dr;
                s_k[pb + i - p0][warp] = kr;
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < p1 - p0; i += PROD_THREADS) {
        uint32_t d = 0, k = 0;
#pragma unroll
        for (int w = 0; w < PROD_THREADS / 32; w++) {
            d += s_d[i][w];
            k += s_k[i][w];
        }
        if (d) atomicAdd(&row_d[p0 + i], d);
        if (k) atomicAdd(&row_k[p0 + i], k);
    }
    if (live)
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (dc[j]) {
                atomicAdd(&col_d[c8 * 8u + j], dc[j]);
                if (kc[j]) atomicAdd(&col_k[c8 * 8u + j], kc[j]);
            }
}

// sum of C(d,2) - C(d-k,2) over the rows and columns
__global__ void k_prod_wsum(const uint32_t *row_d, const uint32_t *row_k, uint32_t a,
                            const uint32_t *col_d, const uint32_t *col_k, uint32_t b,
                            unsigned long long *wedges) {
    unsigned long long w = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a + b; i += gridDim.x * blockDim.x) {
        const uint64_t d = i < a ? row_d[i] : col_d[i - a], k = i < a ? row_k[i] : col_k[i - a];
        w += c2(d) - c2(d - k);
    }
    w = warp_sum_u64(w);
    if (lane_id() == 0 && w) atomicAdd(wedges, w);
}

// c: per product (X X^T, then |X| |X|^T) `split` symmetric ap x ap
// partials; one CTA per row w < a (grid-stride) over the columns w < u < a
__global__ void __launch_bounds__(PROD_THREADS) k_prod_pairs(const float *__restrict__ c,
                                                              uint32_t a, uint32_t ap,
                                                              uint32_t split, CountScratch *sc) {
    const size_t plane = (size_t)ap * ap, half = plane * split;
    unsigned long long bal = 0, tot = 0, cells = 0;
    for (uint32_t w = blockIdx.x; w < a; w += gridDim.x) {
        const float *rd = c + (size_t)w * ap;
        if (threadIdx.x == 0)  // row w's distinct cells: (|X| |X|^T)[w][w]
            for (uint32_t k = 0; k < split; k++) cells += (unsigned long long)rd[half + k * plane + w];
        for (uint32_t u = w + 1 + threadIdx.x; u < a; u += PROD_THREADS) {
            int64_t d = 0, n = 0;  // S - A and S + A: sums of exact integer partials
            for (uint32_t k = 0; k < split; k++) {
                d += (int64_t)rd[k * plane + u];
                n += (int64_t)rd[half + k * plane + u];
            }
            const uint64_t S = (uint64_t)(n + d) >> 1, A = (uint64_t)(n - d) >> 1;
            bal += c2(S) + c2(A);
            tot += c2((uint64_t)n);
        }
        spill_if_large(sc, bal, tot);
    }
    block_sum2<PROD_THREADS>(bal, tot);
    if (threadIdx.x == 0) {
        acc_add(sc, bal, tot);
        if (cells) atomicAdd(&sc->cells, cells);
    }
}

// fewer distinct cells than edges: an edge was listed twice
__global__ void k_prod_check(const CountScratch *sc, int64_t nE, uint32_t *err) {
    if (sc->cells != (unsigned long long)nE) set_error(err, E_DUP);
}

// marks an error word (a failed product launch on a graph built for it alone)
__global__ void k_prod_error(uint32_t *err, uint32_t bits) { set_error(err, bits); }

// One GEMM handle per device, created on the first product count there and
// kept for the process; its stream and workspace are set per call under the
// device's lock (threads share the handle).
constexpr int PROD_MAX_DEVICES = 64;
struct ProdHandle {
    std::once_flag once;
    cublasHandle_t h = nullptr;
    bool ok = false;
    int sms = 1;
    std::mutex mu;
};
ProdHandle g_prod[PROD_MAX_DEVICES];

std::atomic<int> g_prod_mode{0};

// the current device's handle entry, set up once; null if unusable
ProdHandle *prod_handle() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PROD_MAX_DEVICES) {
        cudaGetLastError();
        return nullptr;
    }
    ProdHandle &H = g_prod[dev];
    std::call_once(H.once, [&H, dev]() {
        H.ok = cublasCreate(&H.h) == CUBLAS_STATUS_SUCCESS;
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) H.sms = prop.multiProcessorCount;
        if (cudaFuncSetAttribute(k_prod_fill_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FILL_SMEM) != cudaSuccess)
            H.ok = false;
        cudaGetLastError();
    });
    return H.ok ? &H : nullptr;
}

}  // namespace

bool product_enabled() { return g_prod_mode.load(std::memory_order_relaxed) == 0; }

bool product_ready() { return prod_handle() != nullptr; }

bool launch_product(const DevGraph &g, cudaStream_t s) {
    const ProductPlan &p = g.prod;
    ProdHandle *Hp = p.side >= 0 && g.prod_x && (g.rowptr || !g.product_only) ? prod_handle() : nullptr;
    if (!Hp) {
        if (g.product_only) {  // nothing else can count it
            k_prod_error<<<1, 1, 0, s>>>(g.err, E_INTERNAL);
            note_launch();
        }
        return false;
    }
    ProdHandle &H = *Hp;
    const size_t plane = (size_t)p.ap * p.ld;
    const int ctas = H.sms * 8;
    // 1. X and |X| from the built rows of P (they carry sign flips), or
    // from the input rows when the build stopped at the ranks; windows per
    // row for about six CTAs per SM (at least enough to stay within
    // FILL_WIN columns), 64-column aligned
    FillRows R;
    if (g.product_only) {
        R = FillRows{g.rowptr, g.col, g.sign, nullptr, g.nU};
    } else {
        const SideCSR &P = g.side[p.side];
        R = FillRows{P.off, nullptr, nullptr, P.adj, P.n};
    }
    const bool transpose = g.product_only && p.side == 1;
    uint32_t nwin = (p.ld + FILL_WIN - 1) / FILL_WIN;
    nwin = std::max<uint32_t>(nwin, (6u * H.sms + p.ap - 1) / p.ap);
    uint32_t width = ((p.ld + nwin - 1) / nwin + 63) & ~63u;
    nwin = (p.ld + width - 1) / width;
    if (!transpose && nwin <= FILL_MAX_WINDOWS) {
        k_prod_fill_rows<<<dim3(nwin, p.ap), PROD_THREADS, (size_t)width * sizeof(uint16_t), s>>>(
            R, p.ld, width, plane, g.prod_x);
        note_launch();
    } else {
        cudaMemsetAsync(g.prod_x, 0, 2 * plane * sizeof(uint16_t), s);
        if (R.n > 0 && g.nE > 0) {
            k_prod_fill<<<(int)std::min<int64_t>(R.n, ctas), PROD_THREADS, 0, s>>>(
                R, transpose, p.ld, plane, g.prod_x);
            note_launch();
        }
    }
    // 2. the wedge count, when the build left it to this path
    if (g.product_only) {
        uint32_t *gid = g.prod_cnt, *row_d = gid + p.a + p.b, *row_k = row_d + p.ap;
        uint32_t *col_d = row_k + p.ap, *col_k = col_d + p.ld;
        cudaMemsetAsync(row_d, 0, (2 * (size_t)p.ap + 2 * (size_t)p.ld) * 4, s);
        const SideCSR &P = g.side[p.side], &O = g.side[1 - p.side];
        k_prod_gid<<<std::min<int>((p.a + p.b + PROD_THREADS - 1) / PROD_THREADS, ctas),
                     PROD_THREADS, 0, s>>>(P, O, p.a, p.b, gid);
        note_launch();
        const uint32_t gx = (p.ld / 8 + PROD_THREADS - 1) / PROD_THREADS;
        uint32_t gy = std::max<uint32_t>(1, std::min<uint32_t>(p.a, (4u * H.sms + gx - 1) / gx));
        gy = std::max<uint32_t>(gy, (p.a + DEG_ROWS - 1) / DEG_ROWS);
        const uint32_t rows = (p.a + gy - 1) / gy;  // <= DEG_ROWS
        k_prod_degrees<<<dim3(gx, (p.a + rows - 1) / rows), PROD_THREADS, 0, s>>>(
            g.prod_x + plane, p.a, p.b, p.ld, rows, gid, row_d, row_k, col_d, col_k);
        note_launch();
        k_prod_wsum<<<std::min<int>((p.a + p.b + PROD_THREADS - 1) / PROD_THREADS, ctas),
                      PROD_THREADS, 0, s>>>(row_d, row_k, p.a, col_d, col_k, p.b, g.wedges);
        note_launch();
    }
    // 3. the products, one GEMM per slice of the middles
    cublasStatus_t st;
    {
        std::lock_guard<std::mutex> lk(H.mu);
        st = cublasSetStream(H.h, s);
        if (st == CUBLAS_STATUS_SUCCESS) st = cublasSetWorkspace(H.h, g.prod_ws, p.ws_bytes);
        const float one = 1.0f, zero = 0.0f;
        // column-major view: X (ap rows of ld) is an ld x ap matrix, and
        // op(A) op(B) = X X^T with op(A) = its transpose; slice k of the
        // middles starts k * kc elements into every row
        const size_t cplane = (size_t)p.ap * p.ap;
        for (int m = 0; m < 2 && st == CUBLAS_STATUS_SUCCESS; m++) {
            const uint16_t *xm = g.prod_x + m * plane;
            st = cublasGemmStridedBatchedEx(
                H.h, CUBLAS_OP_T, CUBLAS_OP_N, (int)p.ap, (int)p.ap, (int)p.kc, &one, xm,
                CUDA_R_16BF, (int)p.ld, (long long)p.kc, xm, CUDA_R_16BF, (int)p.ld,
                (long long)p.kc, &zero, g.prod_c + m * p.split * cplane, CUDA_R_32F,
                (int)p.ap, (long long)cplane, (int)p.split, CUBLAS_COMPUTE_32F,
                CUBLAS_GEMM_DEFAULT);
        }
    }
    if (st != CUBLAS_STATUS_SUCCESS) {
        if (g.product_only) {
            k_prod_error<<<1, 1, 0, s>>>(g.err, E_INTERNAL);
            note_launch();
        }
        return false;
    }
    // 4. the pairs, and the duplicate check
    k_prod_pairs<<<std::min<int>((int)p.a, ctas), PROD_THREADS, 0, s>>>(g.prod_c, p.a, p.ap,
                                                                       p.split, g.scratch);
    note_launch();
    k_prod_check<<<1, 1, 0, s>>>(g.scratch, g.nE, g.err);
    note_launch();
    return true;
}

}  // namespace bb

extern "C" int bb_set_matrix_product(int mode) {
    if (mode != 0 && mode != 1) return -1;
    return bb::g_prod_mode.exchange(mode);
}

extern "C" int bb_matrix_product_plan(int64_t nU, int64_t nV, int64_t nE) {
    if (nU < 0 || nV < 0 || nE < 0) return -1;
    return bb::product_plan(nU, nV, nE).side >= 0 && bb::product_enabled() ? 1 : 0;
}
