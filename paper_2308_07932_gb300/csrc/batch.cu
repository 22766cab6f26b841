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
    std::vector<int> size_cls;           // each member's size class
    // re-classification: device scratch (classification temp, then the
    // gathered class counters and statistics), allocated on first use
    void *cmem = nullptr;
    size_t cbytes = 0;
};

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// public tune (kernel order dense, CTA-hash, team, warp) <-> class order
constexpr int KERNEL_CLS[BB_NKERNELS] = {CLS_DENSE, CLS_CTAH, CLS_TEAM, CLS_WARP};

static_assert(BB_NSIZE == NSIZE, "size classes");

// checks t and converts it (kernel order dense, CTA-hash, team, warp ->
// class order; public shapes -> classification parameters)
bb_status to_internal(const bb_batch_tune &t, BatchTune *out) {
    if (t.warp_chunk < 1 || t.warp_chunk > 1024)
        return fail(BB_ERR_INVALID_ARG, "warp_chunk %u outside [1, 1024]", t.warp_chunk);
    if (t.concurrent > 1) return fail(BB_ERR_INVALID_ARG, "concurrent must be 0 or 1");
    if (t.dense_staged > 1) return fail(BB_ERR_INVALID_ARG, "dense_staged must be 0 or 1");
    for (int k = 0; k < BB_NKERNELS; k++)
        if (!(t.grid_frac[k] > 0.f && t.grid_frac[k] <= 1.f))
            return fail(BB_ERR_INVALID_ARG, "grid_frac[%d] outside (0, 1]", k);
    BatchTune T;
    T.warp_chunk = t.warp_chunk;
    T.concurrent = t.concurrent;
    T.dense_staged = t.dense_staged;
    for (int k = 0; k < BB_NKERNELS; k++) T.grid_frac[KERNEL_CLS[k]] = t.grid_frac[k];
    for (int k = 0; k < NSIZE; k++) {
        bb_status st = shape_params(&t.shape[k], &T.shape[k]);
        if (st != BB_OK) return st;
    }
    *out = T;
    return BB_OK;
}

bb_batch_tune to_public(const BatchTune &T) {
    bb_batch_tune t;
    t.warp_chunk = T.warp_chunk;
    t.concurrent = T.concurrent;
    t.dense_staged = T.dense_staged;
    for (int k = 0; k < BB_NKERNELS; k++) t.grid_frac[k] = T.grid_frac[KERNEL_CLS[k]];
    for (int k = 0; k < NSIZE; k++) t.shape[k] = shape_public(T.shape[k]);
    return t;
}

bool same_params(const ClassifyParams &a, const ClassifyParams &b) {
    return a.warp_w_max == b.warp_w_max && a.warp_small_w == b.warp_small_w &&
           a.team_w_max == b.team_w_max && a.split_wedges == b.split_wedges;
}

// class item prefixes over the members (from their host class counters),
// uploaded; the per-class item totals and work statistics updated
bb_status rebuild_prefix(bb_batch *b) {
    const uint32_t n = b->n;
    std::vector<uint32_t> prefix((size_t)NCLS * (n + 1));
    for (int c = 0; c < NCLS; c++) {
        uint64_t acc = 0;
        for (uint32_t i = 0; i < n; i++) {
            prefix[(size_t)c * (n + 1) + i] = (uint32_t)acc;
            acc += b->graphs[i]->g.h_ctr[c];
        }
        if (acc >= UINT32_MAX)
            return fail(BB_ERR_TOO_LARGE, "batch has %llu items of one class (limit 2^32-1)",
                        (unsigned long long)acc);
        prefix[(size_t)c * (n + 1) + n] = (uint32_t)acc;
        b->L.items[c] = (uint32_t)acc;
    }
    for (int k = 0; k < 3 * NCLS; k++) b->cls_stats[k] = 0;
    for (uint32_t i = 0; i < n; i++)
        for (int k = 0; k < 3 * NCLS; k++) b->cls_stats[k] += b->graphs[i]->g.h_cls_stats[k];
    cudaStream_t s = b->ctx->stream;
    BB_CUDA(cudaMemcpyAsync((void *)b->L.prefix, prefix.data(), prefix.size() * 4,
                            cudaMemcpyHostToDevice, s), "copy class prefixes");
    // the host vector must outlive the copy
    return wait_bounded(s, "class prefixes");
}

// gives every member its size class's bucket shape (re-classifying those
// whose shape changes) and rebuilds the class prefixes
bb_status apply_shapes(bb_batch *b, const BatchTune &T) {
    bb_ctx *ctx = b->ctx;
    cudaStream_t s = ctx->stream;
    std::vector<uint32_t> todo;
    for (uint32_t i = 0; i < b->n; i++)
        if (!same_params(b->graphs[i]->g.cls, T.shape[b->size_cls[i]])) todo.push_back(i);
    if (todo.empty()) return BB_OK;
    if (!b->cmem) {
        size_t tmp = 0;
        for (bb_graph *g : b->graphs) tmp = std::max(tmp, classify_temp_bytes(g->g.nU, g->g.nV));
        b->cbytes = align256(tmp) + align256((size_t)b->n * NCTR * 4) +
                    align256((size_t)b->n * 3 * NCLS * 8);
        bb_status st = dev_alloc(ctx, &b->cmem, b->cbytes, "batch re-classification");
        if (st != BB_OK) { b->cmem = nullptr; return st; }
    }
    size_t tmp = 0;
    for (bb_graph *g : b->graphs) tmp = std::max(tmp, classify_temp_bytes(g->g.nU, g->g.nV));
    char *p = (char *)b->cmem;
    uint32_t *d_ctr = (uint32_t *)(p + align256(tmp));
    unsigned long long *d_stats =
        (unsigned long long *)(p + align256(tmp) + align256((size_t)b->n * NCTR * 4));
    for (uint32_t i : todo) {
        DevGraph &g = b->graphs[i]->g;
        g.cls = T.shape[b->size_cls[i]];
        classify_graph(g, b->cmem, s);  // one after another on s: the scratch is shared
    }
    BB_CUDA(cudaGetLastError(), "re-classification");
    launch_batch_classes(b->L, d_ctr, d_stats, s);
    BB_CUDA(cudaGetLastError(), "class counter gather");
    bb_status st = wait_bounded(s, "re-classification");
    if (st != BB_OK) return st;
    std::vector<uint32_t> h_ctr((size_t)b->n * NCTR);
    std::vector<unsigned long long> h_stats((size_t)b->n * 3 * NCLS);
    BB_CUDA(cudaMemcpy(h_ctr.data(), d_ctr, h_ctr.size() * 4, cudaMemcpyDeviceToHost),
            "copy class counters");
    BB_CUDA(cudaMemcpy(h_stats.data(), d_stats, h_stats.size() * 8, cudaMemcpyDeviceToHost),
            "copy class statistics");
    for (uint32_t i = 0; i < b->n; i++) {
        DevGraph &g = b->graphs[i]->g;
        memcpy(g.h_ctr, &h_ctr[(size_t)i * NCTR], sizeof(g.h_ctr));
        memcpy(g.h_cls_stats, &h_stats[(size_t)i * 3 * NCLS], sizeof(g.h_cls_stats));
    }
    return rebuild_prefix(b);
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
    b->size_cls.resize((size_t)n);
    for (int64_t i = 0; i < n; i++) b->size_cls[i] = size_class(graphs[i]->g.nE);
    const size_t b_graphs = align256(sizeof(DevGraph) * (size_t)n);
    const size_t b_prefix = align256((size_t)NCLS * (n + 1) * 4);
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
    if (e != cudaSuccess) { bb_batch_free(b); return cuda_fail(e, "batch set-up"); }
    // the host arrays above must stay alive until the copies are done
    st = wait_bounded(s, "batch set-up");
    // members whose shape differs from their size class's default shape are
    // re-classified; then the class prefixes
    if (st == BB_OK) st = apply_shapes(b, b->tune);
    if (st == BB_OK) st = rebuild_prefix(b);
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
    BatchTune T;
    bb_status st = to_internal(*tune, &T);
    if (st != BB_OK) return st;
    std::lock_guard<std::mutex> lk(b->ctx->mu);
    if ((st = set_device(b->ctx)) != BB_OK) return st;
    drop_exec(b);  // recaptured with the new shapes on the next count
    if ((st = apply_shapes(b, T)) != BB_OK) return st;
    b->tune = T;
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
    // the dense walker, then each size class's bucket shape, one knob at a time
    for (uint32_t staged = 0; staged < 2 && st == BB_OK; staged++) {
        if (staged == best.dense_staged || b->L.items[CLS_DENSE] == 0) continue;
        BatchTune T = best;
        T.dense_staged = staged;
        double ms;
        if ((st = time_of(T, &ms)) == BB_OK && ms < best_ms) { best = T; best_ms = ms; }
    }
    bool have[NSIZE] = {};
    for (int c : b->size_cls) have[c] = true;
    const uint32_t small_w[] = {0, 16, 32, 96};
    const uint32_t warp_w[] = {2048, 8192, 16384};
    const uint32_t team_w[] = {4096, 16384};
    const uint32_t split_w[] = {16384, 65536, 262144};
    for (int k = 0; k < NSIZE && st == BB_OK; k++) {
        if (!have[k]) continue;
        auto tryp = [&](const ClassifyParams &p) {
            if (st != BB_OK || same_params(p, best.shape[k])) return;
            BatchTune T = best;
            T.shape[k] = p;
            double ms;
            if ((st = apply_shapes(b, T)) != BB_OK) return;
            if ((st = time_of(T, &ms)) == BB_OK && ms < best_ms) { best = T; best_ms = ms; }
        };
        for (uint32_t v : small_w) {
            ClassifyParams p = best.shape[k];
            p.warp_small_w = std::min(v, p.warp_w_max);
            tryp(p);
        }
        for (uint32_t v : warp_w) {
            ClassifyParams p = best.shape[k];
            p.warp_w_max = v;
            p.warp_small_w = std::min(p.warp_small_w, v);
            tryp(p);
        }
        for (uint32_t v : team_w) {
            ClassifyParams p = best.shape[k];
            p.team_w_max = v;
            tryp(p);
        }
        for (uint32_t v : split_w) {
            ClassifyParams p = best.shape[k];
            p.split_wedges = v;
            tryp(p);
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st == BB_OK) st = apply_shapes(b, best);
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
    dev_free(ctx, b->cmem, b->cbytes);
    delete b;
}

}  // extern "C"
