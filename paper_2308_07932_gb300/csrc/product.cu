// product.cu - the matrix-product path for graphs with a small dense side
// (the plan and its exactness argument are in graph.cuh).
//
// Per pair (w, u) of the pair side P, over the middles v of the other side:
// S = #{v : sign(w,v) sign(v,u) = +1} and A = #{v : = -1} are the pair's
// symmetric and asymmetric wedge tallies (Defs. 5-6), and by Lemma 2 the
// pair lies in C(S,2) + C(A,2) balanced and C(S+A,2) butterflies in all.
// With X the signed adjacency (X[w][v] = sign(w,v), 0 for no edge),
// (X X^T)[w][u] = S - A and (|X| |X|^T)[w][u] = S + A. Three steps on the
// caller's stream:
//   k_prod_fill   writes X and |X| (bf16, rows = P's side ranks, columns =
//                 the other side's ranks) from the built sign-packed rows;
//   two strided-batched GEMMs (cuBLAS, bf16 in, fp32 sums) form both
//                 products, each as a batch of partial products over
//                 slices of the middles (ProductPlan::split);
//   k_prod_pairs  adds each pair's partials (in integers) and sums
//                 C(S,2) + C(A,2) and C(S+A,2) over the pairs w < u into the
//                 128-bit accumulators of the wedge classes.
#include <cublas_v2.h>

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
constexpr int PROD_THREADS = 256;

// one CTA per row of P (grid-stride): entry x = column << 1 | negative
__global__ void __launch_bounds__(PROD_THREADS) k_prod_fill(SideCSR P, uint32_t ld,
                                                             size_t plane, uint16_t *x) {
    for (int64_t r = blockIdx.x; r < P.n; r += gridDim.x) {
        const int64_t b = P.off[r], e = P.off[r + 1];
        uint16_t *row = x + (size_t)r * ld;
        for (int64_t p = b + threadIdx.x; p < e; p += PROD_THREADS) {
            const uint32_t ent = P.adj[p];
            const uint32_t c = ent >> 1;
            row[c] = (ent & 1u) ? BF16_MINUS_ONE : BF16_PLUS_ONE;
            row[plane + c] = BF16_PLUS_ONE;
        }
    }
}

// c: per product (X X^T, then |X| |X|^T) `split` symmetric a x a partials;
// one CTA per row w (grid-stride) over the columns u > w
__global__ void __launch_bounds__(PROD_THREADS) k_prod_pairs(const float *__restrict__ c,
                                                              uint32_t a, uint32_t split,
                                                              CountScratch *sc) {
    const size_t plane = (size_t)a * a, half = plane * split;
    unsigned long long bal = 0, tot = 0;
    for (uint32_t w = blockIdx.x; w < a; w += gridDim.x) {
        const float *rd = c + (size_t)w * a;
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
    if (threadIdx.x == 0) acc_add(sc, bal, tot);
}

// One GEMM handle per device, created on the first product count there and
// kept for the process; its stream and workspace are set per call under the
// device's lock (threads share the handle).
constexpr int PROD_MAX_DEVICES = 64;
struct ProdHandle {
    std::once_flag once;
    cublasHandle_t h = nullptr;
    bool ok = false;
    std::mutex mu;
};
ProdHandle g_prod[PROD_MAX_DEVICES];
int g_prod_sms[PROD_MAX_DEVICES];

std::atomic<int> g_prod_mode{0};

}  // namespace

bool product_enabled() { return g_prod_mode.load(std::memory_order_relaxed) == 0; }

bool launch_product(const DevGraph &g, cudaStream_t s) {
    const ProductPlan &p = g.prod;
    if (p.side < 0 || !g.prod_x) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PROD_MAX_DEVICES) {
        cudaGetLastError();
        return false;
    }
    ProdHandle &H = g_prod[dev];
    std::call_once(H.once, [&H, dev]() {
        H.ok = cublasCreate(&H.h) == CUBLAS_STATUS_SUCCESS;
        cudaDeviceProp prop;
        g_prod_sms[dev] = cudaGetDeviceProperties(&prop, dev) == cudaSuccess
                              ? prop.multiProcessorCount : 1;
        cudaGetLastError();
    });
    if (!H.ok) return false;
    const size_t plane = (size_t)p.a * p.ld;
    const int grid = (int)std::min<int64_t>(p.a, (int64_t)g_prod_sms[dev] * 8);
    cudaMemsetAsync(g.prod_x, 0, 2 * plane * sizeof(uint16_t), s);
    k_prod_fill<<<grid, PROD_THREADS, 0, s>>>(g.side[p.side], p.ld, plane, g.prod_x);
    note_launch();
    cublasStatus_t st;
    {
        std::lock_guard<std::mutex> lk(H.mu);
        st = cublasSetStream(H.h, s);
        if (st == CUBLAS_STATUS_SUCCESS) st = cublasSetWorkspace(H.h, g.prod_ws, p.ws_bytes);
        const float one = 1.0f, zero = 0.0f;
        // column-major view: X (a rows of ld) is an ld x a matrix, and
        // op(A) op(B) = X X^T with op(A) = its transpose; slice k of the
        // middles starts k * kc elements into every row
        const size_t cplane = (size_t)p.a * p.a;
        for (int m = 0; m < 2 && st == CUBLAS_STATUS_SUCCESS; m++) {
            const uint16_t *xm = g.prod_x + m * plane;
            st = cublasGemmStridedBatchedEx(
                H.h, CUBLAS_OP_T, CUBLAS_OP_N, (int)p.a, (int)p.a, (int)p.kc, &one, xm,
                CUDA_R_16BF, (int)p.ld, (long long)p.kc, xm, CUDA_R_16BF, (int)p.ld,
                (long long)p.kc, &zero, g.prod_c + m * p.split * cplane, CUDA_R_32F, (int)p.a,
                (long long)cplane, (int)p.split, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
        }
    }
    if (st != CUBLAS_STATUS_SUCCESS) return false;
    k_prod_pairs<<<grid, PROD_THREADS, 0, s>>>(g.prod_c, p.a, p.split, g.scratch);
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
