// runtime.h - host-side state behind the C ABI (contexts, resident graphs)
// and the helpers the ABI's translation units share: error reporting,
// bounded waits and budgeted device allocation.
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <mutex>

#include "../../include/bb.h"
#include "graph.cuh"

namespace bb {

struct Engine;  // serving engine (serve.cu)

// results copied back after a count or a build
struct HostResult {
    unsigned long long acc[4];
    uint32_t count_err;
    uint32_t build_err;
    unsigned long long wedges;
    unsigned long long cls_stats[3 * NCLS];
    uint32_t ctr[NCTR];
};

constexpr int NEV = 7;  // build begin/end, count kernel boundaries (5)

}  // namespace bb

struct bb_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    cudaStream_t own = nullptr, stream = nullptr;
    bb::BuildAux aux{};  // the build's auxiliary stream and fork/join events
    // one-shot workspace
    void *ws_graph = nullptr;
    size_t ws_graph_cap = 0;
    void *ws_temp = nullptr;
    size_t ws_temp_cap = 0;
    void *ws_in = nullptr;  // device copies of host inputs (bb_count_csr)
    size_t ws_in_cap = 0;
    int64_t *ws_pv = nullptr;  // device per-vertex output for host requests
    size_t ws_pv_cap = 0;
    void *ws_pe = nullptr;     // per-edge output and entry accumulators
    size_t ws_pe_cap = 0;
    void *ws_flip = nullptr;   // incremental re-count: edge list, records, flags
    size_t ws_flip_cap = 0;
    void *ws_base = nullptr;   // BB-Base: per-CTA group buffers
    size_t ws_base_cap = 0;
    bb::DevGraph oneshot;
    int64_t layout_key[3] = {-1, -1, -1};
    // the one-shot path's work after validation, captured as a CUDA graph
    // for one shape and set of buffers (key) and replayed while they repeat
    cudaGraphExec_t step_exec = nullptr;
    const void *step_key[11] = {};   // key of step_exec
    const void *step_last[11] = {};  // key of the previous call (capture when it repeats)
    uint64_t step_launches = 0;     // kernels in the captured graph
    bb::HostResult *h_res = nullptr;  // pinned
    // host inputs: rowptr and edge-chunk copy events (copies run on the
    // second auxiliary stream while the first chunks are checked)
    cudaEvent_t in_ev[1 + bb::StagedInput::MAX_CHUNKS] = {};
    std::mutex mu;
    bool timing = false;
    cudaEvent_t ev[bb::NEV] = {};
    bool have_build_ev = false;
    // the last count (and the captured step) took the matrix-product path
    bool last_product = false, step_product = false;
    bb_timing last = {};
    bb::Engine *engine = nullptr;  // started by bb_ctx_serve or the first bb_submit
    // bucket shape of later builds (bb_ctx_set_shape) and its version (part
    // of the step graph's key)
    bb::ClassifyParams shape;
    bool dense_staged = false;
    uint64_t shape_version = 0;
};

struct bb_graph {
    bb_ctx *ctx = nullptr;
    bb::DevGraph g;
    void *mem = nullptr;
    size_t bytes = 0;
    void *raw = nullptr;
    size_t raw_bytes = 0;
    // counts of the current signs, when known (the base of incremental re-counts)
    bool have_counts = false;
    int64_t last_balanced = 0, last_total = 0;
};

namespace bb {

// sets the calling thread's bb_last_error() text; returns st
bb_status fail(bb_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
bb_status cuda_fail(cudaError_t e, const char *what);
// waits for the work queued so far on s; BB_ERR_TIMEOUT after the limit
bb_status wait_bounded(cudaStream_t s, const char *what);
// cudaMalloc within the context's budget (BB_ERR_BUDGET / BB_ERR_OOM)
bb_status dev_alloc(bb_ctx *ctx, void **p, size_t bytes, const char *what);
void dev_free(bb_ctx *ctx, void *p, size_t bytes);
bb_status set_device(bb_ctx *ctx);
bb_status map_build_error(uint32_t e);
// argument checks of a CSR given to the library (sizes, NULLs, id limits)
bb_status check_csr(const bb_csr *csr, const int8_t *signs);
// a public bucket shape (NULL = defaults) as classification parameters,
// BB_ERR_INVALID_ARG outside its ranges
bb_status shape_params(const bb_class_shape *shape, ClassifyParams *out);
// the public form of classification parameters
bb_class_shape shape_public(const ClassifyParams &p);
// stops the context's serving engine (waits for running requests)
void engine_stop(bb_ctx *ctx);
// adds launches made by replaying a captured CUDA graph to bb_launch_count;
// retract_launches takes back those counted while capturing (not run then)
void note_launches(uint64_t n);
void retract_launches(uint64_t n);
uint64_t launches();

}  // namespace bb

// Named host ranges for timeline profilers (NVTX; header-only, a no-op
// unless a profiler is attached): one per public call and build stage.
namespace bb {
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace bb

#define BB_CUDA(call, what)                                      \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return bb::cuda_fail(e_, what);   \
    } while (0)
