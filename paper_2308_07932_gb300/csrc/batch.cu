// batch.cu - bb_batch_*: many resident graphs counted by one persistent
// kernel per work class, captured once as a CUDA graph and replayed, plus
// the autotuner that picks the per-class launch shapes.
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "runtime.h"

using namespace bb;

struct bb_batch {
    bb_ctx *ctx = nullptr;
    std::vector<bb_graph *> graphs;
    uint32_t n = 0;
    // device: graph descriptors, class prefixes, cursors, results
    void *mem = nullptr;
    size_t bytes = 0;
    BatchLaunch L{};
    unsigned long long cls_stats[3 * NCLS] = {};  // summed over the members
    unsigned long long *h_out = nullptr;  // pinned [n * BATCH_OUT]
    BatchTune tune;
    cudaStream_t side[NCLS - 1] = {};
    cudaEvent_t ev[NCLS] = {};
    cudaGraphExec_t exec = nullptr;
    cudaStream_t exec_stream = nullptr;  // stream the graph was captured on
    uint64_t exec_launches = 0;          // kernels in one replay
};

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// public tune (kernel order dense, CTA-hash, team, warp) <-> class order
constexpr int KERNEL_CLS[BB_NKERNELS] = {CLS_DENSE, CLS_CTAH, CLS_TEAM, CLS_WARP};

bb_status check_tune(const bb_batch_tune &t) {
    if (t.warp_chunk < 1 || t.warp_chunk > 1024)
        return fail(BB_ERR_INVALID_ARG, "warp_chunk %u outside [1, 1024]", t.warp_chunk);
    if (t.concurrent > 1) return fail(BB_ERR_INVALID_ARG, "concurrent must be 0 or 1");
    for (int k = 0; k < BB_NKERNELS; k++)
        if (!(t.grid_frac[k] > 0.f && t.grid_frac[k] <= 1.f))
            return fail(BB_ERR_INVALID_ARG, "grid_frac[%d] outside (0, 1]", k);
    return BB_OK;
}

BatchTune to_internal(const bb_batch_tune &t) {
    BatchTune T;
    T.warp_chunk = t.warp_chunk;
    T.concurrent = t.concurrent;
    for (int k = 0; k < BB_NKERNELS; k++) T.grid_frac[KERNEL_CLS[k]] = t.grid_frac[k];
    return T;
}

bb_batch_tune to_public(const BatchTune &T) {
    bb_batch_tune t;
    t.warp_chunk = T.warp_chunk;
    t.concurrent = T.concurrent;
    for (int k = 0; k < BB_NKERNELS; k++) t.grid_frac[k] = T.grid_frac[KERNEL_CLS[k]];
    return t;
}

void drop_exec(bb_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_stream = nullptr;
}

// queue one batched count (uncaptured) on the context's stream
bb_status launch_direct(bb_batch *b, const BatchTune &T) {
    launch_count_batch(b->L, T, b->ctx->stream, b->side, b->ev);
    BB_CUDA(cudaGetLastError(), "batch launch");
    return BB_OK;
}

// capture reset + class kernels + gather + copy-back as one CUDA graph
bb_status capture(bb_batch *b) {
    drop_exec(b);
    cudaStream_t s = b->ctx->stream;
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return fail(BB_ERR_INVALID_ARG, "a batch needs a context stream other than the default stream");
    BB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    const uint64_t before = launches();
    launch_count_batch(b->L, b->tune, s, b->side, b->ev);
    cudaMemcpyAsync(b->h_out, b->L.out, (size_t)b->n * BATCH_OUT * 8, cudaMemcpyDeviceToHost, s);
    const uint64_t in_graph = launches() - before;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "capture"); }
    // launches made while capturing were recorded, not run
    note_launches((uint64_t)0 - in_graph);
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->exec = nullptr; return cuda_fail(e, "graph instantiate"); }
    b->exec_stream = s;
    b->exec_launches = in_graph;
    return BB_OK;
}

}  // namespace

extern "C" {

bb_status bb_batch_create(bb_ctx *ctx, bb_graph *const *graphs, int64_t n, bb_batch **out) {
    if (!ctx || !out || (n > 0 && !graphs)) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (n < 1 || n > (1 << 24)) return fail(BB_ERR_INVALID_ARG, "batch of %lld graphs", (long long)n);
    for (int64_t i = 0; i < n; i++) {
        if (!graphs[i]) return fail(BB_ERR_INVALID_ARG, "graph %lld is NULL", (long long)i);
        if (graphs[i]->ctx != ctx)
            return fail(BB_ERR_INVALID_ARG, "graph %lld belongs to another context", (long long)i);
    }
    {  // each graph once: members accumulate into their own graph's scratch
        std::vector<bb_graph *> sorted(graphs, graphs + n);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return fail(BB_ERR_INVALID_ARG, "a graph is listed twice in the batch");
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    bb_batch *b = new (std::nothrow) bb_batch();
    if (!b) return fail(BB_ERR_OOM, "host allocation failed");
    b->ctx = ctx;
    b->n = (uint32_t)n;
    b->graphs.assign(graphs, graphs + n);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3 * NCLS; k++) b->cls_stats[k] += graphs[i]->g.h_cls_stats[k];
    // class item prefixes over the graphs
    std::vector<uint32_t> prefix((size_t)NCLS * (n + 1));
    for (int c = 0; c < NCLS; c++) {
        uint64_t acc = 0;
        for (int64_t i = 0; i < n; i++) {
            prefix[(size_t)c * (n + 1) + i] = (uint32_t)acc;
            acc += graphs[i]->g.h_ctr[c];
        }
        if (acc >= UINT32_MAX) {
            delete b;
            return fail(BB_ERR_TOO_LARGE, "batch has %llu items of one class (limit 2^32-1)",
                        (unsigned long long)acc);
        }
        prefix[(size_t)c * (n + 1) + n] = (uint32_t)acc;
        b->L.items[c] = (uint32_t)acc;
    }
    const size_t b_graphs = align256(sizeof(DevGraph) * (size_t)n);
    const size_t b_prefix = align256(prefix.size() * 4);
    const size_t b_next = 256;
    const size_t b_out = align256((size_t)n * BATCH_OUT * 8);
    b->bytes = b_graphs + b_prefix + b_next + b_out;
    st = dev_alloc(ctx, &b->mem, b->bytes, "batch");
    if (st != BB_OK) { delete b; return st; }
    char *p = (char *)b->mem;
    b->L.graphs = (const DevGraph *)p;
    b->L.prefix = (const uint32_t *)(p + b_graphs);
    b->L.next = (uint32_t *)(p + b_graphs + b_prefix);
    b->L.out = (unsigned long long *)(p + b_graphs + b_prefix + b_next);
    b->L.n = b->n;
    std::vector<DevGraph> descs((size_t)n);
    for (int64_t i = 0; i < n; i++) descs[i] = graphs[i]->g;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMallocHost((void **)&b->h_out, (size_t)n * BATCH_OUT * 8);
    if (e != cudaSuccess) { b->h_out = nullptr; bb_batch_free(b); return cuda_fail(e, "cudaMallocHost"); }
    for (int k = 0; k < NCLS - 1 && e == cudaSuccess; k++)
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
    for (int k = 0; k < NCLS && e == cudaSuccess; k++)
        e = cudaEventCreateWithFlags(&b->ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)b->L.graphs, descs.data(), sizeof(DevGraph) * (size_t)n,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)b->L.prefix, prefix.data(), prefix.size() * 4,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { bb_batch_free(b); return cuda_fail(e, "batch set-up"); }
    // the host arrays above must stay alive until the copies are done
    st = wait_bounded(s, "batch set-up");
    if (st != BB_OK) { bb_batch_free(b); return st; }
    *out = b;
    return BB_OK;
}

bb_status bb_batch_count(bb_batch *b, int64_t *balanced, int64_t *total, bb_status *status_opt) {
    bb::Range range_("bb batch count");
    if (!b || !balanced || !total) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_ctx *ctx = b->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    if (ctx->timing) {
        // traced count: uncaptured, classes one after another between events
        launch_count_batch(b->L, b->tune, ctx->stream, b->side, b->ev, ctx->ev + 2);
        BB_CUDA(cudaGetLastError(), "batch launch");
        BB_CUDA(cudaMemcpyAsync(b->h_out, b->L.out, (size_t)b->n * BATCH_OUT * 8,
                                cudaMemcpyDeviceToHost, ctx->stream), "copy batch results");
        if ((st = wait_bounded(ctx->stream, "batch count")) != BB_OK) return st;
        bb_timing &T = ctx->last;
        T = bb_timing{};
        float ms = 0;
        for (int k = 0; k < BB_NKERNELS; k++)
            if (cudaEventElapsedTime(&ms, ctx->ev[2 + k], ctx->ev[3 + k]) == cudaSuccess)
                T.kernel_ms[k] = ms;
        if (cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[2 + BB_NKERNELS]) == cudaSuccess)
            T.count_ms = ms;
        for (int k = 0; k < BB_NKERNELS; k++) {
            T.wedges[k] = (int64_t)b->cls_stats[KERNEL_CLS[k]];
            T.middles[k] = (int64_t)b->cls_stats[NCLS + KERNEL_CLS[k]];
            T.anchors[k] = (int64_t)b->cls_stats[2 * NCLS + KERNEL_CLS[k]];
        }
        cudaGetLastError();
    } else {
        if (!b->exec || b->exec_stream != ctx->stream)
            if ((st = capture(b)) != BB_OK) return st;
        BB_CUDA(cudaGraphLaunch(b->exec, ctx->stream), "batch graph launch");
        note_launches(b->exec_launches);
        if ((st = wait_bounded(ctx->stream, "batch count")) != BB_OK) return st;
    }
    bb_status first = BB_OK;
    int64_t first_i = -1;
    for (uint32_t i = 0; i < b->n; i++) {
        const unsigned long long *o = b->h_out + (size_t)i * BATCH_OUT;
        const uint32_t cerr = (uint32_t)o[4], berr = (uint32_t)(o[4] >> 32);
        bb_status gs = BB_OK;
        if (berr || cerr) gs = BB_ERR_CUDA;
        else if (o[1] || o[3] || o[0] > (unsigned long long)LLONG_MAX ||
                 o[2] > (unsigned long long)LLONG_MAX)
            gs = BB_ERR_OVERFLOW;
        balanced[i] = gs == BB_OK ? (int64_t)o[0] : -1;
        total[i] = gs == BB_OK ? (int64_t)o[2] : -1;
        if (status_opt) status_opt[i] = gs;
        if (gs != BB_OK && first == BB_OK) { first = gs; first_i = i; }
    }
    if (first == BB_ERR_OVERFLOW)
        return fail(first, "graph %lld: butterfly count exceeds int64", (long long)first_i);
    if (first != BB_OK)
        return fail(first, "graph %lld: internal device check failed", (long long)first_i);
    return BB_OK;
}

bb_status bb_batch_set_tune(bb_batch *b, const bb_batch_tune *tune) {
    if (!b || !tune) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_status st = check_tune(*tune);
    if (st != BB_OK) return st;
    std::lock_guard<std::mutex> lk(b->ctx->mu);
    b->tune = to_internal(*tune);
    drop_exec(b);  // recaptured with the new shapes on the next count
    return BB_OK;
}

bb_status bb_batch_get_tune(const bb_batch *b, bb_batch_tune *out) {
    if (!b || !out) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    *out = to_public(b->tune);
    return BB_OK;
}

bb_status bb_batch_autotune(bb_batch *b, int reps, bb_batch_tune *best_opt, double *best_ms_opt) {
    if (!b) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    if (reps < 1 || reps > 100) return fail(BB_ERR_INVALID_ARG, "reps %d outside [1, 100]", reps);
    bb_ctx *ctx = b->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    cudaStream_t s = ctx->stream;
    cudaEvent_t t0, t1;
    BB_CUDA(cudaEventCreate(&t0), "event");
    if (cudaEventCreate(&t1) != cudaSuccess) { cudaEventDestroy(t0); return cuda_fail(cudaGetLastError(), "event"); }
    // median of reps timed runs of one candidate
    auto time_of = [&](const BatchTune &T, double *ms_out) -> bb_status {
        std::vector<double> v;
        for (int r = 0; r < reps; r++) {
            cudaEventRecord(t0, s);
            bb_status e2 = launch_direct(b, T);
            if (e2 != BB_OK) return e2;
            cudaEventRecord(t1, s);
            if ((e2 = wait_bounded(s, "autotune")) != BB_OK) return e2;
            float ms = 0;
            BB_CUDA(cudaEventElapsedTime(&ms, t0, t1), "event time");
            v.push_back(ms);
        }
        std::sort(v.begin(), v.end());
        *ms_out = v[v.size() / 2];
        return BB_OK;
    };
    BatchTune best = b->tune;
    double best_ms = 0;
    st = launch_direct(b, best);  // warm-up
    if (st == BB_OK) st = wait_bounded(s, "autotune");
    if (st == BB_OK) st = time_of(best, &best_ms);
    // coordinate descent: one knob at a time, keep what helps
    const uint32_t chunks[] = {1, 2, 4, 8, 16, 32, 64};
    const float fracs[] = {0.25f, 0.5f, 0.75f, 1.0f};
    for (int pass = 0; pass < 2 && st == BB_OK; pass++) {
        for (uint32_t c : chunks) {
            if (st != BB_OK || c == best.warp_chunk) continue;
            BatchTune T = best;
            T.warp_chunk = c;
            double ms;
            if ((st = time_of(T, &ms)) == BB_OK && ms < best_ms) { best = T; best_ms = ms; }
        }
        for (uint32_t conc = 0; conc < 2 && st == BB_OK; conc++) {
            if (conc == best.concurrent) continue;
            BatchTune T = best;
            T.concurrent = conc;
            double ms;
            if ((st = time_of(T, &ms)) == BB_OK && ms < best_ms) { best = T; best_ms = ms; }
        }
        for (int c = 0; c < NCLS && st == BB_OK; c++) {
            if (b->L.items[c] == 0) continue;
            for (float f : fracs) {
                if (st != BB_OK || f == best.grid_frac[c]) continue;
                BatchTune T = best;
                T.grid_frac[c] = f;
                double ms;
                if ((st = time_of(T, &ms)) == BB_OK && ms < best_ms) { best = T; best_ms = ms; }
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != BB_OK) return st;
    b->tune = best;
    drop_exec(b);
    if (best_opt) *best_opt = to_public(best);
    if (best_ms_opt) *best_ms_opt = best_ms;
    return BB_OK;
}

void bb_batch_free(bb_batch *b) {
    if (!b) return;
    bb_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    // work still running after the wait limit: its memory is left (leaked)
    // rather than freed under it
    bool idle = wait_bounded(ctx->stream, "batch free") == BB_OK;
    for (int k = 0; k < NCLS - 1 && idle; k++)
        if (b->side[k]) idle = wait_bounded(b->side[k], "batch free") == BB_OK;
    if (!idle) {
        delete b;
        return;
    }
    drop_exec(b);
    for (int k = 0; k < NCLS - 1; k++)
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
    for (int k = 0; k < NCLS; k++)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->h_out) cudaFreeHost(b->h_out);
    dev_free(ctx, b->mem, b->bytes);
    delete b;
}

}  // extern "C"
