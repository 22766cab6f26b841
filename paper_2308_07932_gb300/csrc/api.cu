// api.cu - the C ABI declared in include/bb.h: contexts, device memory
// budget, one-shot counts, resident graphs, errors.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace bb;

namespace {
std::atomic<uint64_t> g_launches{0};
thread_local std::string t_err;
// limit of a bounded wait on device work
std::atomic<double> g_timeout_s{600.0};
}  // namespace

void bb::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void bb::note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void bb::retract_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
uint64_t bb::launches() { return g_launches.load(std::memory_order_relaxed); }

bb_status bb::fail(bb_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

bb_status bb::cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear sticky-free errors
    return fail(BB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Waits for all work queued so far on `s`, polling an event so that a stuck
// device turns into BB_ERR_TIMEOUT instead of a hang of the caller.
bb_status bb::wait_bounded(cudaStream_t s, const char *what) {
    cudaEvent_t ev;
    BB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    cudaError_t e = cudaEventRecord(ev, s);
    if (e != cudaSuccess) { cudaEventDestroy(ev); return cuda_fail(e, what); }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return cuda_fail(e, what); }
        double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        const double limit = g_timeout_s.load(std::memory_order_relaxed);
        if (dt > limit) {
            cudaEventDestroy(ev);
            return fail(BB_ERR_TIMEOUT, "%s: device work did not finish within %g s", what, limit);
        }
        // poll without sleeping for the first millisecond (short device
        // work, such as the input validation, then ends within a few
        // microseconds of its completion), then every 20 us
        if (dt > 1e-3) std::this_thread::sleep_for(std::chrono::microseconds(20));
        else std::this_thread::yield();
    }
    cudaEventDestroy(ev);
    return BB_OK;
}

bb_status bb::shape_params(const bb_class_shape *shape, ClassifyParams *out) {
    ClassifyParams p;
    if (shape) {
        if (shape->warp_w_max < 1 || shape->warp_w_max > WARP_W_MAX)
            return fail(BB_ERR_INVALID_ARG, "warp_w_max %u outside [1, %llu]", shape->warp_w_max,
                        (unsigned long long)WARP_W_MAX);
        if (shape->warp_small_w > shape->warp_w_max)
            return fail(BB_ERR_INVALID_ARG, "warp_small_w %u above warp_w_max %u",
                        shape->warp_small_w, shape->warp_w_max);
        if (shape->team_w_max < 1 || shape->team_w_max > TEAM_W_MAX)
            return fail(BB_ERR_INVALID_ARG, "team_w_max %u outside [1, %llu]", shape->team_w_max,
                        (unsigned long long)TEAM_W_MAX);
        if (shape->split_wedges < 1024 || shape->split_wedges > (1u << 30))
            return fail(BB_ERR_INVALID_ARG, "split_wedges %u outside [1024, 2^30]",
                        shape->split_wedges);
        p.warp_w_max = shape->warp_w_max;
        p.warp_small_w = shape->warp_small_w;
        p.team_w_max = shape->team_w_max;
        p.split_wedges = shape->split_wedges;
    }
    *out = p;
    return BB_OK;
}

bb_class_shape bb::shape_public(const ClassifyParams &p) {
    bb_class_shape s;
    s.warp_w_max = p.warp_w_max;
    s.warp_small_w = p.warp_small_w;
    s.team_w_max = p.team_w_max;
    s.split_wedges = p.split_wedges;
    return s;
}

// The same bound without creating anything (no event): polls the stream
// until it is idle. For paths that must not create CUDA objects.
bb_status bb::wait_stream_bounded(cudaStream_t s, const char *what) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return BB_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, what);
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        const double limit = g_timeout_s.load(std::memory_order_relaxed);
        if (dt > limit)
            return fail(BB_ERR_TIMEOUT, "%s: device work did not finish within %g s", what, limit);
        if (dt > 1e-3) std::this_thread::sleep_for(std::chrono::microseconds(20));
        else std::this_thread::yield();
    }
}

bb_status bb::check_csr(const bb_csr *csr, const int8_t *signs) {
    if (!csr) return fail(BB_ERR_INVALID_ARG, "csr is NULL");
    if (csr->nU < 0 || csr->nV < 0 || csr->nE < 0)
        return fail(BB_ERR_INVALID_ARG, "negative size (nU=%lld nV=%lld nE=%lld)",
                    (long long)csr->nU, (long long)csr->nV, (long long)csr->nE);
    if (csr->nU + csr->nV >= ((int64_t)1 << 31))
        return fail(BB_ERR_TOO_LARGE, "nU + nV = %lld must be below 2^31",
                    (long long)(csr->nU + csr->nV));
    if (csr->nE >= ((int64_t)1 << 32) - 1)
        return fail(BB_ERR_TOO_LARGE, "nE = %lld must be below 2^32 - 1", (long long)csr->nE);
    if (csr->nU == 0 && csr->nE != 0)
        return fail(BB_ERR_INVALID_ARG, "nE must be 0 when nU is 0");
    if (!csr->rowptr) return fail(BB_ERR_INVALID_ARG, "rowptr is NULL");
    if (csr->nE > 0 && (!csr->col || !signs))
        return fail(BB_ERR_INVALID_ARG, "col or signs is NULL");
    return BB_OK;
}

bb_status bb::map_build_error(uint32_t e) {
    if (e & E_ROWPTR) return fail(BB_ERR_INVALID_ARG, "rowptr is not a valid CSR row pointer");
    if (e & E_COL) return fail(BB_ERR_INVALID_ARG, "a column id is outside [0, nV)");
    if (e & E_SIGN) return fail(BB_ERR_INVALID_ARG, "a sign is not +1 or -1");
    if (e & E_DUP) return fail(BB_ERR_INVALID_ARG, "an edge is listed twice");
    if (e) return fail(BB_ERR_CUDA, "internal device check failed (0x%x)", e);
    return BB_OK;
}

// lets other translation units of the library set bb_last_error()
bb_status bb::report_error(bb_status st, const char *msg) { return fail(st, "%s", msg); }

namespace {
// allocations left until the injected failure (0 = none armed)
std::atomic<int64_t> g_alloc_fail_in{0};
}

bb_status bb::dev_alloc(bb_ctx *ctx, void **p, size_t bytes, const char *what) {
    if (bytes == 0) bytes = 256;
    if (ctx->used + bytes > ctx->budget)
        return fail(BB_ERR_BUDGET, "%s: %zu bytes would exceed the budget (%llu of %llu used)",
                    what, bytes, (unsigned long long)ctx->used, (unsigned long long)ctx->budget);
    for (int64_t k = g_alloc_fail_in.load(); k > 0;) {
        if (g_alloc_fail_in.compare_exchange_weak(k, k - 1)) {
            if (k == 1) {
                *p = nullptr;
                return fail(BB_ERR_OOM, "%s: cudaMalloc(%zu) failed (injected failure)", what,
                            bytes);
            }
            break;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(BB_ERR_OOM, "%s: cudaMalloc(%zu) failed: %s", what, bytes,
                    cudaGetErrorString(e));
    }
    ctx->used += bytes;
    return BB_OK;
}

void bb::dev_free(bb_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    if (bytes == 0) bytes = 256;
    ctx->used -= bytes;
}

bb_status bb::set_device(bb_ctx *ctx) {
    BB_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    return BB_OK;
}

namespace {

// grow-only workspace buffer
bb_status ensure(bb_ctx *ctx, void **buf, size_t *cap, size_t need, const char *what) {
    if (*cap >= need && *buf) return BB_OK;
    // the old buffer may still be in use by queued work
    bb_status ws = wait_bounded(ctx->stream, "workspace sync");
    if (ws != BB_OK) return ws;
    dev_free(ctx, *buf, *cap);
    *buf = nullptr;
    *cap = 0;
    size_t want = need + need / 8;  // headroom so slightly larger graphs reuse it
    bb_status st = dev_alloc(ctx, buf, want, what);
    if (st != BB_OK) {
        st = dev_alloc(ctx, buf, need, what);
        if (st != BB_OK) return st;
        want = need;
    }
    *cap = want;
    return BB_OK;
}

// reads back results and maps device-side errors
bb_status finish_count(bb_ctx *ctx, const DevGraph &g, cudaStream_t s, int64_t *balanced,
                       int64_t *total, int64_t *wedges_opt) {
    HostResult *h = ctx->h_res;
    BB_CUDA(cudaMemcpyAsync(h->acc, g.scratch->acc, sizeof(h->acc), cudaMemcpyDeviceToHost, s),
            "copy counts");
    BB_CUDA(cudaMemcpyAsync(&h->count_err, &g.scratch->err, 4, cudaMemcpyDeviceToHost, s),
            "copy count status");
    BB_CUDA(cudaMemcpyAsync(&h->build_err, g.err, 4, cudaMemcpyDeviceToHost, s),
            "copy build status");
    BB_CUDA(cudaMemcpyAsync(&h->wedges, g.wedges, 8, cudaMemcpyDeviceToHost, s), "copy wedges");
    if (ctx->timing)
        BB_CUDA(cudaMemcpyAsync(h->cls_stats, g.cls_stats, sizeof(h->cls_stats),
                                cudaMemcpyDeviceToHost, s), "copy class stats");
    bb_status st = wait_bounded(s, "count");
    if (st != BB_OK) return st;
    BB_CUDA(cudaGetLastError(), "count kernels");
    if (ctx->timing) {
        bb_timing &T = ctx->last;
        T = bb_timing{};
        float ms = 0;
        if (ctx->have_build_ev && cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess)
            T.build_ms = ms;
        for (int k = 0; k < BB_NKERNELS; k++)
            if (cudaEventElapsedTime(&ms, ctx->ev[2 + k], ctx->ev[3 + k]) == cudaSuccess)
                T.kernel_ms[k] = ms;
        if (cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[2 + BB_NKERNELS]) == cudaSuccess)
            T.count_ms = ms;
        const int order[BB_NKERNELS] = {CLS_DENSE, CLS_CTAH, CLS_TEAM, CLS_WARP};
        for (int k = 0; k < BB_NKERNELS; k++) {
            T.wedges[k] = (int64_t)h->cls_stats[order[k]];
            T.middles[k] = (int64_t)h->cls_stats[NCLS + order[k]];
            T.anchors[k] = (int64_t)h->cls_stats[2 * NCLS + order[k]];
        }
        if (ctx->last_product) {  // ev[0] .. ev[1] spans the product path
            T.product_ms = T.kernel_ms[0];
            for (int k = 0; k < BB_NKERNELS; k++) {
                T.kernel_ms[k] = 0;
                T.wedges[k] = T.middles[k] = T.anchors[k] = 0;
            }
        }
        cudaGetLastError();
    }
    if (h->build_err) return map_build_error(h->build_err);
    if (h->count_err) return fail(BB_ERR_CUDA, "internal count check failed (0x%x)", h->count_err);
    if (h->acc[1] || h->acc[3] || h->acc[0] > (unsigned long long)LLONG_MAX ||
        h->acc[2] > (unsigned long long)LLONG_MAX)
        return fail(BB_ERR_OVERFLOW, "butterfly count exceeds int64");
    *balanced = (int64_t)h->acc[0];
    *total = (int64_t)h->acc[2];
    if (wedges_opt) *wedges_opt = (int64_t)h->wedges;
    return BB_OK;
}

// The one-shot path's work after validation (the rest of the build and the
// count) as one CUDA graph: captured when a call repeats the previous one's
// shape, input buffers, workspaces and timing setting, and replayed while
// they repeat, so the ~60 launches of a step cost one (a one-off call
// launches directly and pays no capture). Returns false (nothing launched)
// when the call is not a repeat or the stream cannot be captured; the
// caller launches directly then.
bool replay_step(bb_ctx *ctx, DevGraph &g, const bb_csr *csr, const int8_t *signs,
                 bool product_only) {
    // the degree sort's key width depends on the inputs' largest degree
    const void *key[11] = {(const void *)(intptr_t)csr->nU, (const void *)(intptr_t)csr->nV,
                           (const void *)(intptr_t)csr->nE, csr->rowptr, csr->col, signs,
                           ctx->ws_temp, ctx->ws_graph,
                           (const void *)(intptr_t)(ctx->timing | (product_enabled() ? 2 : 0)),
                           (const void *)(intptr_t)g.deg_bits,
                           (const void *)(intptr_t)ctx->shape_version};
    static_assert(sizeof(key) == sizeof(ctx->step_key), "step key size");
    static_assert(sizeof(key) == sizeof(ctx->step_last), "step key size");
    cudaStream_t s = ctx->stream;
    if (!ctx->step_exec || memcmp(ctx->step_key, key, sizeof(key)) != 0) {
        const bool repeat = memcmp(ctx->step_last, key, sizeof(key)) == 0;
        memcpy(ctx->step_last, key, sizeof(key));
        if (!repeat) return false;
        if (ctx->step_exec) {
            cudaGraphExecDestroy(ctx->step_exec);
            ctx->step_exec = nullptr;
        }
        if (!s || cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        const uint64_t l0 = launches();
        build_rest(g, csr->rowptr, csr->col, signs, ctx->ws_temp, s, &ctx->aux, product_only);
        if (ctx->timing) record_timing_event(ctx->ev[1], s);
        ctx->step_product = launch_count(g, s, ctx->timing ? ctx->ev + 2 : nullptr);
        const uint64_t n = launches() - l0;
        retract_launches(n);  // captured, not run
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        // any call that failed while capturing (its error is pending) voids the graph
        const cudaError_t pending = cudaGetLastError();
        if (e == cudaSuccess && pending == cudaSuccess)
            e = cudaGraphInstantiate(&ctx->step_exec, graph, 0);
        else if (e == cudaSuccess)
            e = pending;
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
            ctx->step_exec = nullptr;
            return false;
        }
        memcpy(ctx->step_key, key, sizeof(key));
        ctx->step_launches = n;
    }
    if (cudaGraphLaunch(ctx->step_exec, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ctx->last_product = ctx->step_product;
    note_launches(ctx->step_launches);
    return true;
}

// one-shot path on device-resident inputs (`in`: still being copied)
bb_status count_device(bb_ctx *ctx, const bb_csr *csr, const int8_t *signs, int64_t *balanced,
                       int64_t *total, int64_t *pv_dev, int64_t *wedges_opt,
                       const StagedInput *in = nullptr) {
    Range range("bb count (device inputs)");
    const int64_t nU = csr->nU, nV = csr->nV, nE = csr->nE;
    BuildSizes bs = build_sizes(nU, nV, nE);
    bb_status st = ensure(ctx, &ctx->ws_graph, &ctx->ws_graph_cap, bs.graph_bytes, "graph workspace");
    if (st != BB_OK) return st;
    st = ensure(ctx, &ctx->ws_temp, &ctx->ws_temp_cap, bs.temp_bytes, "build workspace");
    if (st != BB_OK) return st;
    cudaStream_t s = ctx->stream;
    DevGraph &g = ctx->oneshot;
    bool relayout = ctx->layout_key[0] != nU || ctx->layout_key[1] != nV ||
                    ctx->layout_key[2] != nE;
    layout_graph(g, nU, nV, nE, ctx->ws_graph);
    if (relayout) {
        // split-merge counters must start at zero; counts leave them zeroed
        BB_CUDA(cudaMemsetAsync(g.gpart, 0, (size_t)g.gpart_cap * 4, s), "zero merge buffer");
        BB_CUDA(cudaMemsetAsync(g.gdone, 0, MAX_SPLIT_JOBS * 4, s), "zero merge counters");
        ctx->layout_key[0] = nU; ctx->layout_key[1] = nV; ctx->layout_key[2] = nE;
    }
    if (ctx->timing) BB_CUDA(cudaEventRecord(ctx->ev[0], s), "event");
    g.cls = ctx->shape;
    g.dense_staged = ctx->dense_staged;
    uint32_t verr = 0;
    {
        Range r("validate");
        st = build_validate(g, csr->rowptr, csr->col, signs, ctx->ws_temp, s, in, &verr,
                            &ctx->h_res->build_err, &ctx->h_res->ctr[CTR_MAXDEG]);
    }
    if (st != BB_OK) {
        ctx->layout_key[0] = -1;
        return st;
    }
    if (verr) {
        ctx->layout_key[0] = -1;  // leave the merge buffers to be re-zeroed
        return map_build_error(verr);
    }
    Range r_rest("build and count");
    // a plain count of a graph the matrix-product path takes needs only the
    // ranks and the wedge count from the build; that path reads the inputs
    const bool product_only = !pv_dev && g.prod.side >= 0 && product_enabled() && product_ready();
    g.rowptr = const_cast<int64_t *>(csr->rowptr);
    g.col = const_cast<int32_t *>(csr->col);
    g.sign = const_cast<int8_t *>(signs);
    if (pv_dev || !replay_step(ctx, g, csr, signs, product_only)) {
        build_rest(g, csr->rowptr, csr->col, signs, ctx->ws_temp, s, &ctx->aux, product_only);
        BB_CUDA(cudaGetLastError(), "build kernels");
        if (ctx->timing) BB_CUDA(cudaEventRecord(ctx->ev[1], s), "event");
        cudaEvent_t *ev = ctx->timing ? ctx->ev + 2 : nullptr;
        if (pv_dev) {
            launch_per_vertex(g, pv_dev, s, ev);
            ctx->last_product = false;
        } else {
            ctx->last_product = launch_count(g, s, ev);
        }
    }
    ctx->have_build_ev = ctx->timing;
    BB_CUDA(cudaGetLastError(), "count launch");
    return finish_count(ctx, g, s, balanced, total, wedges_opt);
}

}  // namespace

extern "C" {

const char *bb_last_error(void) { return t_err.c_str(); }

const char *bb_version(void) { return "bb 0.1 (sm_103a)"; }

bb_status bb_ctx_create(int device, uint64_t hbm_budget_bytes, bb_ctx **out) {
    if (!out) return fail(BB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(BB_ERR_NO_DEVICE, "no CUDA device (%s)", cudaGetErrorString(e));
    }
    if (device < 0 || device >= n) return fail(BB_ERR_INVALID_ARG, "device %d of %d", device, n);
    cudaDeviceProp prop;
    BB_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3)
        return fail(BB_ERR_NO_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a",
                    device, prop.major, prop.minor);
    BB_CUDA(cudaSetDevice(device), "cudaSetDevice");
    bb_ctx *ctx = new (std::nothrow) bb_ctx();
    if (!ctx) return fail(BB_ERR_OOM, "host allocation failed");
    ctx->device = device;
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "cudaMemGetInfo"); }
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(free_b * 0.9);
    e = cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "cudaStreamCreate"); }
    ctx->stream = ctx->own;
    e = aux_create(ctx->aux);
    if (e != cudaSuccess) { bb_ctx_destroy(ctx); return cuda_fail(e, "auxiliary streams"); }
    e = cudaMallocHost((void **)&ctx->h_res, sizeof(HostResult));
    if (e != cudaSuccess) { bb_ctx_destroy(ctx); return cuda_fail(e, "cudaMallocHost"); }
    for (int k = 0; k < NEV; k++) {
        e = cudaEventCreate(&ctx->ev[k]);
        if (e != cudaSuccess) { bb_ctx_destroy(ctx); return cuda_fail(e, "cudaEventCreate"); }
    }
    for (cudaEvent_t &ev : ctx->in_ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { bb_ctx_destroy(ctx); return cuda_fail(e, "cudaEventCreate"); }
    }
    count_init();
    *out = ctx;
    return BB_OK;
}

void bb_ctx_destroy(bb_ctx *ctx) {
    if (!ctx) return;
    engine_stop(ctx);
    cudaSetDevice(ctx->device);
    if (wait_bounded(ctx->stream, "context destroy") != BB_OK) {
        // work still running after the wait limit: leave its memory and
        // streams in place (leaked) rather than hang the caller
        delete ctx;
        return;
    }
    if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
    dev_free(ctx, ctx->ws_graph, ctx->ws_graph_cap);
    dev_free(ctx, ctx->ws_temp, ctx->ws_temp_cap);
    dev_free(ctx, ctx->ws_in, ctx->ws_in_cap);
    dev_free(ctx, ctx->ws_pv, ctx->ws_pv_cap);
    dev_free(ctx, ctx->ws_pe, ctx->ws_pe_cap);
    dev_free(ctx, ctx->ws_flip, ctx->ws_flip_cap);
    dev_free(ctx, ctx->ws_base, ctx->ws_base_cap);
    if (ctx->h_res) cudaFreeHost(ctx->h_res);
    for (int k = 0; k < NEV; k++)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    for (cudaEvent_t ev : ctx->in_ev)
        if (ev) cudaEventDestroy(ev);
    aux_destroy(ctx->aux);
    if (ctx->own) cudaStreamDestroy(ctx->own);
    delete ctx;
}

bb_status bb_ctx_set_timing(bb_ctx *ctx, int enable) {
    if (!ctx) return fail(BB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->timing = enable != 0;
    return BB_OK;
}

bb_status bb_ctx_last_timing(const bb_ctx *ctx, bb_timing *out) {
    if (!ctx || !out) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    *out = ctx->last;
    return BB_OK;
}

uint64_t bb_launch_count(void) { return launches(); }

bb_status bb_set_wait_timeout(double seconds) {
    if (!(seconds > 0.0 && seconds <= 86400.0))
        return fail(BB_ERR_INVALID_ARG, "timeout %g s outside (0, 86400]", seconds);
    g_timeout_s.store(seconds, std::memory_order_relaxed);
    return BB_OK;
}

bb_status bb_ctx_set_shape(bb_ctx *ctx, const bb_class_shape *shape, int dense_staged) {
    if (!ctx) return fail(BB_ERR_INVALID_ARG, "NULL context");
    if (dense_staged != 0 && dense_staged != 1)
        return fail(BB_ERR_INVALID_ARG, "dense_staged must be 0 or 1");
    ClassifyParams p;
    bb_status st = shape_params(shape, &p);
    if (st != BB_OK) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->shape = p;
    ctx->dense_staged = dense_staged != 0;
    ctx->shape_version++;
    return BB_OK;
}

bb_status bb_graph_set_shape(bb_graph *G, const bb_class_shape *shape, int dense_staged) {
    if (!G) return fail(BB_ERR_INVALID_ARG, "graph is NULL");
    if (dense_staged != 0 && dense_staged != 1)
        return fail(BB_ERR_INVALID_ARG, "dense_staged must be 0 or 1");
    ClassifyParams p;
    bb_status st = shape_params(shape, &p);
    if (st != BB_OK) return st;
    bb_ctx *ctx = G->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((st = set_device(ctx)) != BB_OK) return st;
    st = ensure(ctx, &ctx->ws_temp, &ctx->ws_temp_cap, classify_temp_bytes(G->g.nU, G->g.nV),
                "build workspace");
    if (st != BB_OK) return st;
    cudaStream_t s = ctx->stream;
    G->g.cls = p;
    G->g.dense_staged = dense_staged != 0;
    classify_graph(G->g, ctx->ws_temp, s);
    BB_CUDA(cudaGetLastError(), "classification");
    BB_CUDA(cudaMemcpyAsync(ctx->h_res->ctr, G->g.ctr, sizeof(ctx->h_res->ctr),
                            cudaMemcpyDeviceToHost, s), "copy class counters");
    BB_CUDA(cudaMemcpyAsync(ctx->h_res->cls_stats, G->g.cls_stats, sizeof(ctx->h_res->cls_stats),
                            cudaMemcpyDeviceToHost, s), "copy class statistics");
    if ((st = wait_bounded(s, "classification")) != BB_OK) return st;
    memcpy(G->g.h_ctr, ctx->h_res->ctr, sizeof(G->g.h_ctr));
    memcpy(G->g.h_cls_stats, ctx->h_res->cls_stats, sizeof(G->g.h_cls_stats));
    return BB_OK;
}

bb_status bb_set_alloc_failure(int64_t nth) {
    if (nth < 0) return fail(BB_ERR_INVALID_ARG, "nth must be >= 0");
    g_alloc_fail_in.store(nth);
    return BB_OK;
}

bb_status bb_ctx_set_stream(bb_ctx *ctx, void *stream) {
    if (!ctx) return fail(BB_ERR_INVALID_ARG, "ctx is NULL");
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own;
    return BB_OK;
}

uint64_t bb_ctx_device_bytes(const bb_ctx *ctx) { return ctx ? ctx->used : 0; }

bb_status bb_count_csr_device(bb_ctx *ctx, const bb_csr *csr_dev, const int8_t *signs_dev,
                              int64_t *balanced, int64_t *total, int64_t *per_vertex_dev_opt,
                              int64_t *wedges_opt) {
    if (!ctx || !balanced || !total) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_status st = check_csr(csr_dev, signs_dev);
    if (st != BB_OK) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((st = set_device(ctx)) != BB_OK) return st;
    return count_device(ctx, csr_dev, signs_dev, balanced, total, per_vertex_dev_opt, wedges_opt);
}

bb_status bb_count_csr(bb_ctx *ctx, const bb_csr *csr, const int8_t *signs, int64_t *balanced,
                       int64_t *total, int64_t *per_vertex_opt, int64_t *wedges_opt) {
    if (!ctx || !balanced || !total) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_status st = check_csr(csr, signs);
    if (st != BB_OK) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((st = set_device(ctx)) != BB_OK) return st;
    Range range("bb count (host inputs)");
    const int64_t nU = csr->nU, nE = csr->nE;
    size_t b_row = ((size_t)(nU + 1) * 8 + 255) & ~(size_t)255;
    size_t b_col = ((size_t)nE * 4 + 255) & ~(size_t)255;
    size_t b_sg = ((size_t)nE + 255) & ~(size_t)255;
    st = ensure(ctx, &ctx->ws_in, &ctx->ws_in_cap, b_row + b_col + b_sg + 256, "input workspace");
    if (st != BB_OK) return st;
    char *p = (char *)ctx->ws_in;
    bb_csr d = *csr;
    d.rowptr = (const int64_t *)p;
    d.col = (const int32_t *)(p + b_row);
    const int8_t *dsg = (const int8_t *)(p + b_row + b_col);
    cudaStream_t s = ctx->stream;
    // copies on the second auxiliary stream (the staging buffers are free:
    // the previous call has finished), in edge chunks of at least 2^21
    // whose checks start as each chunk lands
    cudaStream_t cs = ctx->aux.stream2;
    StagedInput in;
    in.chunks = nE > 0 ? (int)std::min<int64_t>(StagedInput::MAX_CHUNKS / 2, (nE >> 21) + 1) : 0;
    for (int c = 0; c <= in.chunks; c++) in.lo[c] = nE * c / std::max(in.chunks, 1);
    BB_CUDA(cudaMemcpyAsync((void *)d.rowptr, csr->rowptr, (size_t)(nU + 1) * 8,
                            cudaMemcpyHostToDevice, cs), "copy rowptr");
    BB_CUDA(cudaEventRecord(ctx->in_ev[0], cs), "input event");
    in.rowptr_ready = ctx->in_ev[0];
    for (int c = 0; c < in.chunks; c++) {
        const int64_t lo = in.lo[c], n = in.lo[c + 1] - lo;
        if (n > 0) {
            BB_CUDA(cudaMemcpyAsync((void *)(d.col + lo), csr->col + lo, (size_t)n * 4,
                                    cudaMemcpyHostToDevice, cs), "copy col");
            BB_CUDA(cudaMemcpyAsync((void *)(dsg + lo), signs + lo, (size_t)n,
                                    cudaMemcpyHostToDevice, cs), "copy signs");
        }
        BB_CUDA(cudaEventRecord(ctx->in_ev[1 + c], cs), "input event");
        in.ready[c] = ctx->in_ev[1 + c];
    }
    int64_t *pv_dev = nullptr;
    if (per_vertex_opt) {
        size_t need = (size_t)(csr->nU + csr->nV) * 8;
        st = ensure(ctx, (void **)&ctx->ws_pv, &ctx->ws_pv_cap, need, "per-vertex workspace");
        if (st != BB_OK) return st;
        pv_dev = ctx->ws_pv;
    }
    st = count_device(ctx, &d, dsg, balanced, total, pv_dev, wedges_opt, &in);
    if (st != BB_OK) return st;
    if (per_vertex_opt) {
        BB_CUDA(cudaMemcpyAsync(per_vertex_opt, pv_dev, (size_t)(csr->nU + csr->nV) * 8,
                                cudaMemcpyDeviceToHost, s), "copy per-vertex");
        st = wait_bounded(s, "per-vertex copy");
    }
    return st;
}

// ------------------------------------------------------- resident graphs
static bb_status upload_impl(bb_ctx *ctx, const bb_csr *csr, const int8_t *signs, bool on_device,
                             bb_graph **out) {
    bb::Range range_("bb graph upload");
    if (!ctx || !out) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    bb_status st = check_csr(csr, signs);
    if (st != BB_OK) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((st = set_device(ctx)) != BB_OK) return st;
    const int64_t nU = csr->nU, nV = csr->nV, nE = csr->nE;
    BuildSizes bs = build_sizes(nU, nV, nE);
    bb_graph *G = new (std::nothrow) bb_graph();
    if (!G) return fail(BB_ERR_OOM, "host allocation failed");
    G->ctx = ctx;
    size_t b_row = ((size_t)(nU + 1) * 8 + 255) & ~(size_t)255;
    size_t b_col = ((size_t)nE * 4 + 255) & ~(size_t)255;
    size_t b_sg = ((size_t)nE + 255) & ~(size_t)255;
    G->raw_bytes = b_row + b_col + b_sg + 256;
    st = dev_alloc(ctx, &G->raw, G->raw_bytes, "graph input copy");
    if (st != BB_OK) { delete G; return st; }
    st = dev_alloc(ctx, &G->mem, bs.graph_bytes, "graph");
    if (st != BB_OK) { dev_free(ctx, G->raw, G->raw_bytes); delete G; return st; }
    G->bytes = bs.graph_bytes;
    st = ensure(ctx, &ctx->ws_temp, &ctx->ws_temp_cap, bs.temp_bytes, "build workspace");
    if (st != BB_OK) { bb_graph_free(G); return st; }
    cudaStream_t s = ctx->stream;
    char *p = (char *)G->raw;
    G->g.rowptr = (int64_t *)p;
    G->g.col = (int32_t *)(p + b_row);
    G->g.sign = (int8_t *)(p + b_row + b_col);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(G->g.rowptr, csr->rowptr, (size_t)(nU + 1) * 8, kind, s);
    if (e == cudaSuccess && nE > 0) e = cudaMemcpyAsync(G->g.col, csr->col, (size_t)nE * 4, kind, s);
    if (e == cudaSuccess && nE > 0) e = cudaMemcpyAsync(G->g.sign, signs, (size_t)nE, kind, s);
    if (e != cudaSuccess) { bb_graph_free(G); return cuda_fail(e, "copy graph"); }
    int64_t *rp = G->g.rowptr;
    int32_t *cl = G->g.col;
    int8_t *sg = G->g.sign;
    layout_graph(G->g, nU, nV, nE, G->mem);
    G->g.rowptr = rp; G->g.col = cl; G->g.sign = sg;
    G->g.cls = ctx->shape;
    G->g.dense_staged = ctx->dense_staged;
    cudaMemsetAsync(G->g.gpart, 0, (size_t)G->g.gpart_cap * 4, s);
    cudaMemsetAsync(G->g.gdone, 0, MAX_SPLIT_JOBS * 4, s);
    uint32_t verr = 0;
    st = build_graph(G->g, rp, cl, sg, ctx->ws_temp, s, &ctx->aux, &verr);
    if (st != BB_OK) { bb_graph_free(G); return st; }
    if (verr) { bb_graph_free(G); return map_build_error(verr); }
    e = cudaMemcpyAsync(&ctx->h_res->build_err, G->g.err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctx->h_res->wedges, G->g.wedges, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_res->ctr, G->g.ctr, sizeof(ctx->h_res->ctr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_res->cls_stats, G->g.cls_stats, sizeof(ctx->h_res->cls_stats),
                            cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) { bb_graph_free(G); return cuda_fail(e, "copy build status"); }
    st = wait_bounded(s, "graph build");
    if (st != BB_OK) { bb_graph_free(G); return st; }
    if (ctx->h_res->build_err) {
        uint32_t be = ctx->h_res->build_err;
        bb_graph_free(G);
        return map_build_error(be);
    }
    G->g.h_wedges = ctx->h_res->wedges;
    memcpy(G->g.h_ctr, ctx->h_res->ctr, sizeof(G->g.h_ctr));
    memcpy(G->g.h_cls_stats, ctx->h_res->cls_stats, sizeof(G->g.h_cls_stats));
    *out = G;
    return BB_OK;
}

bb_status bb_graph_upload(bb_ctx *ctx, const bb_csr *csr, const int8_t *signs, bb_graph **out) {
    return upload_impl(ctx, csr, signs, false, out);
}

bb_status bb_graph_upload_device(bb_ctx *ctx, const bb_csr *csr_dev, const int8_t *signs_dev,
                                 bb_graph **out) {
    return upload_impl(ctx, csr_dev, signs_dev, true, out);
}

bb_status bb_count(bb_graph *G, int64_t *balanced, int64_t *total, int64_t *per_vertex_opt) {
    bb::Range range_("bb count (resident graph)");
    if (!G || !balanced || !total) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_ctx *ctx = G->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    ctx->have_build_ev = false;
    int64_t *pv_dev = nullptr;
    if (per_vertex_opt) {
        const size_t need = (size_t)(G->g.nU + G->g.nV) * 8;
        st = ensure(ctx, (void **)&ctx->ws_pv, &ctx->ws_pv_cap, need, "per-vertex workspace");
        if (st != BB_OK) return st;
        pv_dev = ctx->ws_pv;
    }
    cudaEvent_t *ev = ctx->timing ? ctx->ev + 2 : nullptr;
    if (pv_dev) {
        launch_per_vertex(G->g, pv_dev, ctx->stream, ev);
        ctx->last_product = false;
    } else {
        ctx->last_product = launch_count(G->g, ctx->stream, ev);
    }
    BB_CUDA(cudaGetLastError(), "count launch");
    st = finish_count(ctx, G->g, ctx->stream, balanced, total, nullptr);
    if (st == BB_OK) {
        G->have_counts = true;
        G->last_balanced = *balanced;
        G->last_total = *total;
    }
    if (st != BB_OK || !pv_dev) return st;
    BB_CUDA(cudaMemcpyAsync(per_vertex_opt, pv_dev, (size_t)(G->g.nU + G->g.nV) * 8,
                            cudaMemcpyDeviceToHost, ctx->stream), "copy per-vertex");
    return wait_bounded(ctx->stream, "per-vertex copy");
}

bb_status bb_count_edges(bb_graph *G, int64_t *per_edge, int64_t *balanced_opt,
                         int64_t *total_opt) {
    bb::Range range_("bb count per edge");
    if (!G || !per_edge) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_ctx *ctx = G->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    ctx->have_build_ev = false;
    const int64_t nE = G->g.nE;
    const size_t b_out = ((size_t)nE * 8 + 255) & ~(size_t)255;
    st = ensure(ctx, &ctx->ws_pe, &ctx->ws_pe_cap, b_out + (size_t)nE * 16 + 256,
                "per-edge workspace");
    if (st != BB_OK) return st;
    int64_t *out_dev = (int64_t *)ctx->ws_pe;
    unsigned long long *acc = (unsigned long long *)((char *)ctx->ws_pe + b_out);
    cudaStream_t s = ctx->stream;
    launch_per_edge(G->g, out_dev, acc, s, ctx->timing ? ctx->ev + 2 : nullptr);
    ctx->last_product = false;
    BB_CUDA(cudaGetLastError(), "per-edge launch");
    int64_t b = 0, t = 0;
    st = finish_count(ctx, G->g, s, &b, &t, nullptr);
    if (st != BB_OK) return st;
    G->have_counts = true;
    G->last_balanced = b;
    G->last_total = t;
    if (nE > 0)
        BB_CUDA(cudaMemcpyAsync(per_edge, out_dev, (size_t)nE * 8, cudaMemcpyDeviceToHost, s),
                "copy per-edge");
    st = wait_bounded(s, "per-edge copy");
    if (st != BB_OK) return st;
    if (balanced_opt) *balanced_opt = b;
    if (total_opt) *total_opt = t;
    return BB_OK;
}

bb_status bb_count_flipped(bb_graph *G, const int64_t *edge_idx, int64_t n, int64_t *balanced,
                           int64_t *total, int *incremental_opt) {
    bb::Range range_("bb count flipped");
    if (!G || !balanced || !total || n < 0 || (n > 0 && !edge_idx))
        return fail(BB_ERR_INVALID_ARG, "bad argument");
    const int64_t nE = G->g.nE;
    for (int64_t i = 0; i < n; i++)
        if (edge_idx[i] < 0 || edge_idx[i] >= nE)
            return fail(BB_ERR_INVALID_ARG, "edge index %lld outside [0, %lld)",
                        (long long)edge_idx[i], (long long)nE);
    // An edge listed twice flips back. The incremental walk needs each
    // flipped edge once (the edges listed an odd number of times); a recount
    // takes the list as it is. Sets of more than nE/1024 flips are always
    // recounted: on power-law graphs their enumeration exceeds a recount.
    const bool small = n <= nE / 1024;
    std::vector<int64_t> odd;
    if (small) {
        std::vector<int64_t> list(edge_idx, edge_idx + n);
        std::sort(list.begin(), list.end());
        for (size_t i = 0; i < list.size();) {
            size_t j = i;
            while (j < list.size() && list[j] == list[i]) j++;
            if ((j - i) & 1) odd.push_back(list[i]);
            i = j;
        }
    }
    const int64_t m = small ? (int64_t)odd.size() : n;
    const int64_t *flips_host = small ? odd.data() : edge_idx;
    bb_ctx *ctx = G->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    ctx->have_build_ev = false;
    cudaStream_t s = ctx->stream;
    const size_t b_list = ((size_t)(m > 0 ? m : 1) * 8 + 255) & ~(size_t)255;
    st = ensure(ctx, &ctx->ws_flip, &ctx->ws_flip_cap, b_list + 256 + flip_ws_bytes(nE, m),
                "flip workspace");
    if (st != BB_OK) return st;
    int64_t *d_list = (int64_t *)ctx->ws_flip;
    unsigned long long *d_acc = (unsigned long long *)((char *)ctx->ws_flip + b_list);  // cost, up, down
    void *ws = (char *)ctx->ws_flip + b_list + 256;
    if (m > 0)
        BB_CUDA(cudaMemcpyAsync(d_list, flips_host, (size_t)m * 8, cudaMemcpyHostToDevice, s),
                "copy flip list");
    // Enumeration steps (a binary search each, at random places) cost about
    // 16 to 20 times a wedge of the full count on the 2M x 500k graph. A
    // graph the matrix-product path counts is recounted (on the 500 x 50k
    // vote graph 10 flipped edges took 23 ms to walk, a recount 0.16 ms).
    const bool by_product = G->g.prod.side >= 0 && product_enabled();
    bool incremental = false;
    if (G->have_counts && m > 0 && small && !by_product) {
        launch_flip_estimate(G->g, d_list, m, ws, d_acc, s);
        BB_CUDA(cudaGetLastError(), "flip estimate");
        BB_CUDA(cudaMemcpyAsync(ctx->h_res->acc, d_acc, 8, cudaMemcpyDeviceToHost, s), "copy estimate");
        if ((st = wait_bounded(s, "flip estimate")) != BB_OK) return st;
        incremental = ctx->h_res->acc[0] <= G->g.h_wedges / 16;
    }
    G->have_counts = G->have_counts && (incremental || m == 0);
    if (incremental) {
        launch_flip_delta(G->g, m, ws, d_acc + 1, s);
        BB_CUDA(cudaGetLastError(), "flip delta");
        BB_CUDA(cudaMemcpyAsync(ctx->h_res->acc + 1, d_acc + 1, 16, cudaMemcpyDeviceToHost, s),
                "copy delta");
    }
    if (m > 0) {
        launch_flip(G->g, d_list, m, s);
        BB_CUDA(cudaGetLastError(), "sign flip");
    }
    if (incremental || (G->have_counts && m == 0)) {
        if ((st = wait_bounded(s, "incremental count")) != BB_OK) return st;
        if (incremental) {
            const unsigned long long up = ctx->h_res->acc[1], down = ctx->h_res->acc[2];
            const long long d3 = (long long)up - (long long)down;
            if (d3 % 3 != 0) return fail(BB_ERR_CUDA, "internal check failed (weighted change %lld)", d3);
            G->last_balanced += d3 / 3;
        }
    } else {
        int64_t b = 0, t = 0;
        ctx->last_product = launch_count(G->g, s, ctx->timing ? ctx->ev + 2 : nullptr);
        BB_CUDA(cudaGetLastError(), "count launch");
        if ((st = finish_count(ctx, G->g, s, &b, &t, nullptr)) != BB_OK) return st;
        G->have_counts = true;
        G->last_balanced = b;
        G->last_total = t;
    }
    *balanced = G->last_balanced;
    *total = G->last_total;
    if (incremental_opt) *incremental_opt = incremental ? 1 : 0;
    return BB_OK;
}

bb_status bb_count_base(bb_graph *G, int64_t *balanced, int64_t *total) {
    bb::Range range_("bb count base (Algorithm 1)");
    if (!G || !balanced || !total) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    bb_ctx *ctx = G->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    cudaStream_t s = ctx->stream;
    // the largest anchor's wedges bound a CTA's group buffer
    st = ensure(ctx, &ctx->ws_base, &ctx->ws_base_cap, 256, "BB-Base workspace");
    if (st != BB_OK) return st;
    unsigned long long *d_acc = (unsigned long long *)ctx->ws_base;  // [0] max work, [1..2] counts
    launch_max_work(G->g, d_acc, s);
    BB_CUDA(cudaGetLastError(), "max work");
    BB_CUDA(cudaMemcpyAsync(ctx->h_res->acc, d_acc, 8, cudaMemcpyDeviceToHost, s), "copy max work");
    if ((st = wait_bounded(s, "max work")) != BB_OK) return st;
    const uint64_t per_cta = std::max<uint64_t>(ctx->h_res->acc[0], 1);
    const size_t need = 256 + (size_t)base_blocks() * ((per_cta + 255) / 256 * 256);
    st = ensure(ctx, &ctx->ws_base, &ctx->ws_base_cap, need, "BB-Base workspace");
    if (st != BB_OK) return st;
    d_acc = (unsigned long long *)ctx->ws_base;
    launch_base(G->g, (uint8_t *)ctx->ws_base + 256, (per_cta + 255) / 256 * 256, d_acc + 1, s);
    BB_CUDA(cudaGetLastError(), "BB-Base");
    BB_CUDA(cudaMemcpyAsync(ctx->h_res->acc + 1, d_acc + 1, 16, cudaMemcpyDeviceToHost, s), "copy counts");
    BB_CUDA(cudaMemcpyAsync(&ctx->h_res->count_err, &G->g.scratch->err, 4, cudaMemcpyDeviceToHost, s),
            "copy status");
    if ((st = wait_bounded(s, "BB-Base")) != BB_OK) return st;
    if (ctx->h_res->count_err)
        return fail(BB_ERR_CUDA, "internal check failed (0x%x)", ctx->h_res->count_err);
    if (ctx->h_res->acc[1] > (unsigned long long)LLONG_MAX || ctx->h_res->acc[2] > (unsigned long long)LLONG_MAX)
        return fail(BB_ERR_OVERFLOW, "butterfly count exceeds int64");
    *balanced = (int64_t)ctx->h_res->acc[1];
    *total = (int64_t)ctx->h_res->acc[2];
    return BB_OK;
}

bb_status bb_graph_flip_signs(bb_graph *G, const int64_t *edge_idx, int64_t n) {
    if (!G || (n > 0 && !edge_idx) || n < 0) return fail(BB_ERR_INVALID_ARG, "bad argument");
    if (n == 0) return BB_OK;
    for (int64_t i = 0; i < n; i++)
        if (edge_idx[i] < 0 || edge_idx[i] >= G->g.nE)
            return fail(BB_ERR_INVALID_ARG, "edge index %lld outside [0, %lld)",
                        (long long)edge_idx[i], (long long)G->g.nE);
    bb_ctx *ctx = G->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    G->have_counts = false;
    void *d = nullptr;
    st = dev_alloc(ctx, &d, (size_t)n * 8, "flip list");
    if (st != BB_OK) return st;
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(d, edge_idx, (size_t)n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        launch_flip(G->g, (const int64_t *)d, n, s);
        e = cudaGetLastError();
    }
    st = e == cudaSuccess ? wait_bounded(s, "sign flip") : cuda_fail(e, "sign flip");
    dev_free(ctx, d, (size_t)n * 8);
    return st;
}

bb_status bb_graph_bytes(int64_t nU, int64_t nV, int64_t nE, uint64_t *resident_opt,
                         uint64_t *workspace_opt) {
    if (nU < 0 || nV < 0 || nE < 0) return fail(BB_ERR_INVALID_ARG, "negative size");
    const BuildSizes bs = build_sizes(nU, nV, nE);
    if (resident_opt) *resident_opt = bs.graph_bytes;
    if (workspace_opt) *workspace_opt = bs.temp_bytes;
    return BB_OK;
}

bb_status bb_graph_info(const bb_graph *G, int64_t *nU, int64_t *nV, int64_t *nE,
                        int64_t *wedges) {
    if (!G) return fail(BB_ERR_INVALID_ARG, "graph is NULL");
    if (nU) *nU = G->g.nU;
    if (nV) *nV = G->g.nV;
    if (nE) *nE = G->g.nE;
    if (wedges) *wedges = (int64_t)G->g.h_wedges;
    return BB_OK;
}

void bb_graph_free(bb_graph *G) {
    if (!G) return;
    bb_ctx *ctx = G->ctx;
    cudaSetDevice(ctx->device);
    if (wait_bounded(ctx->stream, "graph free") != BB_OK) {
        delete G;  // its device memory may still be read: leaked, not freed
        return;
    }
    dev_free(ctx, G->mem, G->bytes);
    dev_free(ctx, G->raw, G->raw_bytes);
    delete G;
}

}  // extern "C"
