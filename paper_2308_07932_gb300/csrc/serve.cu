// serve.cu - the serving engine behind bb_submit / bb_submit_request /
// bb_poll: a FIFO of requests, worker slots with their own CUDA streams,
// continuous admission against the arena (the HBM budget), and a cache of
// resident graphs keyed by the caller's graph key with least-recently-used
// eviction.
//
// A worker takes the oldest admissible request whenever it is free: a
// request whose graph is in use by another request waits without holding
// back the others, and a request that needs memory the arena cannot give
// even after evicting every idle graph waits for running requests to
// release theirs; later requests that need new memory do not overtake it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "arena.h"
#include "runtime.h"

using namespace bb;
using Clock = std::chrono::steady_clock;

struct bb_ticket_s {
    bool managed = false;
    bb_graph *graph = nullptr;  // caller-owned graph (not managed)
    bb_request req{};
    uint32_t flags = 0;
    std::atomic<int> done{0};
    bb_status st = BB_OK;
    int64_t balanced = 0, total = 0;
    bool incremental = false;  // re-counted through the flipped edges only
    std::string err;
    Clock::time_point t_submit, t_start, t_done;
};

namespace bb {

struct Block {
    size_t off = 0, bytes = 0;
    bool held = false;
};

struct Entry {
    uint64_t key = 0;
    DevGraph g;
    Block graph, raw;
    bool busy = false;
    uint64_t last_use = 0;
    // counts of the current signs, when known (the base of incremental re-counts)
    bool have_counts = false;
    int64_t last_balanced = 0, last_total = 0;
};

struct Plan {
    Entry *entry = nullptr;
    bool fresh = false;  // upload and build before counting
    Block temp, flips;
    bool drop = false;   // remove the entry when done
    bool leak = false;   // device work may still run: keep its memory out of the arena
};

struct Slot {
    cudaStream_t s = nullptr;
    BuildAux aux{};           // the build's auxiliary stream and events
    HostResult *h = nullptr;  // pinned
    std::thread th;
};

struct Engine {
    bb_ctx *ctx = nullptr;
    int device = 0;
    char *arena_mem = nullptr;
    size_t arena_bytes = 0;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<bb_ticket_s *> queue;
    std::unordered_map<uint64_t, Entry *> cache;
    std::unordered_set<bb_graph *> busy_graphs;
    std::vector<Slot> slots;
    bool stop = false;
    int running = 0;
    uint64_t tick = 0;
    bb_serve_stats stats{};
};

}  // namespace bb

namespace {

// Flip sets of at most nE/1024 distinct edges on a graph whose counts are
// known may be re-counted incrementally (flips.cu); their arena block also
// holds the located edges, two flag bitmaps and the change accumulators.
bool flips_small(const Entry *e, int64_t n_flip) {
    return e && e->have_counts && n_flip > 0 && n_flip <= e->g.nE / 1024;
}

size_t flip_block_bytes(const Entry *e, int64_t n_flip) {
    const size_t list = Arena::round((size_t)n_flip * 8);
    return flips_small(e, n_flip) ? list + 256 + flip_ws_bytes(e->g.nE, n_flip) : list;
}

struct RawLayout {
    size_t rowptr, col, sign, total;
};

RawLayout raw_layout(int64_t nU, int64_t nE) {
    RawLayout r;
    r.rowptr = 0;
    r.col = Arena::round((size_t)(nU + 1) * 8);
    r.sign = r.col + Arena::round((size_t)nE * 4);
    r.total = r.sign + Arena::round((size_t)nE);
    return r;
}

// finish a ticket without running it (caller holds the engine lock)
void fail_now(Engine *E, bb_ticket_s *t, bb_status st, const char *msg) {
    t->st = st;
    t->err = msg;
    t->t_start = t->t_done = Clock::now();
    E->stats.failed++;
    t->done.store(1, std::memory_order_release);
}

void release_block(Engine *E, Block &b) {
    if (b.held) E->arena.free(b.off, b.bytes);
    b.held = false;
}

// removes a graph from the cache; `evicted`: made room for another request
void remove_entry(Engine *E, Entry *e, bool evicted) {
    release_block(E, e->graph);
    release_block(E, e->raw);
    E->cache.erase(e->key);
    delete e;
    if (evicted) E->stats.evictions++;
}

Entry *lru_idle(Engine *E, const Entry *keep) {
    Entry *best = nullptr;
    for (auto &kv : E->cache) {
        Entry *e = kv.second;
        if (e->busy || e == keep) continue;
        if (!best || e->last_use < best->last_use) best = e;
    }
    return best;
}

// allocates every block of `want` (sizes in, blocks out) or none of them,
// evicting idle graphs (least recently used first) until they fit
bool alloc_all(Engine *E, std::vector<Block *> want, const Entry *keep) {
    for (;;) {
        size_t i = 0;
        for (; i < want.size(); i++) {
            size_t off;
            if (!E->arena.alloc(want[i]->bytes, &off)) break;
            want[i]->off = off;
            want[i]->held = true;
        }
        if (i == want.size()) return true;
        for (size_t j = 0; j < i; j++) release_block(E, *want[j]);
        Entry *victim = lru_idle(E, keep);
        if (!victim) return false;
        remove_entry(E, victim, true);
    }
}

// oldest admissible request, with its plan (caller holds the lock). A key
// whose earlier request is still queued is not admitted again (same-key
// requests run in arrival order).
bb_ticket_s *pick(Engine *E, Plan &plan) {
    bool memory_blocked = false;
    std::vector<uint64_t> waiting;  // keys with an earlier request left in the queue
    auto skip = [&](uint64_t key) { waiting.push_back(key); };
    auto is_waiting = [&](uint64_t key) {
        return std::find(waiting.begin(), waiting.end(), key) != waiting.end();
    };
    for (auto it = E->queue.begin(); it != E->queue.end();) {
        bb_ticket_s *t = *it;
        if (!t->managed) {
            if (E->busy_graphs.count(t->graph)) { ++it; continue; }
            E->busy_graphs.insert(t->graph);
            E->queue.erase(it);
            return t;
        }
        const bb_request &r = t->req;
        if (is_waiting(r.key)) { ++it; continue; }
        auto ce = E->cache.find(r.key);
        if (ce != E->cache.end()) {
            Entry *e = ce->second;
            if (e->busy) { skip(r.key); ++it; continue; }
            Plan p;
            p.entry = e;
            if (r.n_flip > 0) {
                p.flips.bytes = flip_block_bytes(e, r.n_flip);
                std::vector<Block *> want{&p.flips};
                if (!alloc_all(E, want, e)) {
                    if (E->running == 0) {
                        fail_now(E, t, BB_ERR_BUDGET, "the flip list does not fit the serving arena");
                        it = E->queue.erase(it);
                        continue;
                    }
                    skip(r.key);
                    ++it;
                    continue;
                }
            }
            e->busy = true;
            E->stats.cache_hits++;
            plan = p;
            E->queue.erase(it);
            return t;
        }
        if (!r.csr) {
            fail_now(E, t, BB_ERR_INVALID_ARG, "graph key is not resident and no CSR was given");
            it = E->queue.erase(it);
            continue;
        }
        if (memory_blocked) { skip(r.key); ++it; continue; }  // no overtaking for new memory
        const BuildSizes bs = build_sizes(r.csr->nU, r.csr->nV, r.csr->nE);
        Plan p;
        p.fresh = true;
        Entry tmp;
        tmp.graph.bytes = bs.graph_bytes;
        tmp.raw.bytes = raw_layout(r.csr->nU, r.csr->nE).total;
        p.temp.bytes = bs.temp_bytes;
        p.flips.bytes = r.n_flip > 0 ? (size_t)r.n_flip * 8 : 0;
        const size_t need = Arena::round(tmp.graph.bytes) + Arena::round(tmp.raw.bytes) +
                            Arena::round(p.temp.bytes) + (p.flips.bytes ? Arena::round(p.flips.bytes) : 0);
        if (need > E->arena.capacity()) {
            char msg[160];
            snprintf(msg, sizeof(msg), "graph needs %zu bytes; the serving arena holds %zu", need,
                     E->arena.capacity());
            fail_now(E, t, BB_ERR_BUDGET, msg);
            it = E->queue.erase(it);
            continue;
        }
        std::vector<Block *> want{&tmp.graph, &tmp.raw, &p.temp};
        if (p.flips.bytes) want.push_back(&p.flips);
        if (!alloc_all(E, want, nullptr)) {
            if (E->running == 0) {  // nothing will release memory: it cannot fit
                fail_now(E, t, BB_ERR_BUDGET, "graph does not fit the free serving arena");
                it = E->queue.erase(it);
                continue;
            }
            memory_blocked = true;  // wait for running requests to release memory
            skip(r.key);
            ++it;
            continue;
        }
        Entry *e = new Entry();
        e->key = r.key;
        e->graph = tmp.graph;
        e->raw = tmp.raw;
        e->busy = true;
        E->cache[r.key] = e;
        E->stats.uploads++;
        p.entry = e;
        plan = p;
        E->queue.erase(it);
        return t;
    }
    return nullptr;
}

// copies the count results back and waits; fills the ticket
bb_status count_and_wait(Slot &S, const DevGraph &g, bb_ticket_s *t) {
    launch_count(g, S.s);
    BB_CUDA(cudaGetLastError(), "count launch");
    HostResult *h = S.h;
    BB_CUDA(cudaMemcpyAsync(h->acc, g.scratch->acc, sizeof(h->acc), cudaMemcpyDeviceToHost, S.s),
            "copy counts");
    BB_CUDA(cudaMemcpyAsync(&h->count_err, &g.scratch->err, 4, cudaMemcpyDeviceToHost, S.s),
            "copy count status");
    BB_CUDA(cudaMemcpyAsync(&h->build_err, g.err, 4, cudaMemcpyDeviceToHost, S.s),
            "copy build status");
    BB_CUDA(cudaMemcpyAsync(&h->wedges, g.wedges, 8, cudaMemcpyDeviceToHost, S.s), "copy wedges");
    bb_status st = wait_bounded(S.s, "served count");
    if (st != BB_OK) return st;
    if (h->build_err) return map_build_error(h->build_err);
    if (h->count_err) return fail(BB_ERR_CUDA, "internal count check failed (0x%x)", h->count_err);
    if (h->acc[1] || h->acc[3] || h->acc[0] > (unsigned long long)INT64_MAX ||
        h->acc[2] > (unsigned long long)INT64_MAX)
        return fail(BB_ERR_OVERFLOW, "butterfly count exceeds int64");
    t->balanced = (int64_t)h->acc[0];
    t->total = (int64_t)h->acc[2];
    return BB_OK;
}

bb_status run_managed(Engine *E, Slot &S, bb_ticket_s *t, Plan &plan) {
    bb::Range range_("bb served request");
    Entry *e = plan.entry;
    const bb_request &r = t->req;
    cudaStream_t s = S.s;
    if (plan.fresh) {
        const bb_csr *c = r.csr;
        const RawLayout L = raw_layout(c->nU, c->nE);
        char *raw = E->arena_mem + e->raw.off;
        int64_t *rp = (int64_t *)(raw + L.rowptr);
        int32_t *cl = (int32_t *)(raw + L.col);
        int8_t *sg = (int8_t *)(raw + L.sign);
        BB_CUDA(cudaMemcpyAsync(rp, c->rowptr, (size_t)(c->nU + 1) * 8, cudaMemcpyHostToDevice, s),
                "copy rowptr");
        if (c->nE > 0) {
            BB_CUDA(cudaMemcpyAsync(cl, c->col, (size_t)c->nE * 4, cudaMemcpyHostToDevice, s), "copy col");
            BB_CUDA(cudaMemcpyAsync(sg, r.signs, (size_t)c->nE, cudaMemcpyHostToDevice, s), "copy signs");
        }
        layout_graph(e->g, c->nU, c->nV, c->nE, E->arena_mem + e->graph.off);
        e->g.rowptr = rp;
        e->g.col = cl;
        e->g.sign = sg;
        BB_CUDA(cudaMemsetAsync(e->g.gpart, 0, (size_t)e->g.gpart_cap * 4, s), "zero merge buffer");
        BB_CUDA(cudaMemsetAsync(e->g.gdone, 0, MAX_SPLIT_JOBS * 4, s), "zero merge counters");
        uint32_t verr = 0;
        const bb_status bst =
            build_graph(e->g, rp, cl, sg, E->arena_mem + plan.temp.off, s, &S.aux, &verr);
        if (bst != BB_OK) {
            plan.drop = true;
            return bst;
        }
        BB_CUDA(cudaGetLastError(), "build kernels");
        if (verr) {
            plan.drop = true;
            return map_build_error(verr);
        }
    }
    if (r.n_flip > 0) {
        for (int64_t i = 0; i < r.n_flip; i++)
            if (r.flip_idx[i] < 0 || r.flip_idx[i] >= e->g.nE)
                return fail(BB_ERR_INVALID_ARG, "edge index %lld outside [0, %lld)",
                            (long long)r.flip_idx[i], (long long)e->g.nE);
        char *fb = E->arena_mem + plan.flips.off;
        int64_t *d = (int64_t *)fb;
        if (flips_small(e, r.n_flip)) {
            // distinct flips (an edge listed twice flips back), then the
            // incremental walk when it is cheaper than a recount
            std::vector<int64_t> list(r.flip_idx, r.flip_idx + r.n_flip), odd;
            std::sort(list.begin(), list.end());
            for (size_t i = 0; i < list.size();) {
                size_t j = i;
                while (j < list.size() && list[j] == list[i]) j++;
                if ((j - i) & 1) odd.push_back(list[i]);
                i = j;
            }
            const int64_t m = (int64_t)odd.size();
            unsigned long long *acc = (unsigned long long *)(fb + Arena::round((size_t)r.n_flip * 8));
            void *ws = (char *)acc + 256;
            if (m > 0) {
                BB_CUDA(cudaMemcpyAsync(d, odd.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s),
                        "copy flip list");
                launch_flip_estimate(e->g, d, m, ws, acc, s);
                BB_CUDA(cudaGetLastError(), "flip estimate");
                BB_CUDA(cudaMemcpyAsync(S.h->acc, acc, 8, cudaMemcpyDeviceToHost, s), "copy estimate");
                bb_status st = wait_bounded(s, "flip estimate");
                if (st != BB_OK) return st;
            }
            if (m == 0 || S.h->acc[0] <= e->g.h_wedges / 16) {
                if (m > 0) {
                    launch_flip_delta(e->g, m, ws, acc + 1, s);
                    BB_CUDA(cudaGetLastError(), "flip delta");
                    BB_CUDA(cudaMemcpyAsync(S.h->acc + 1, acc + 1, 16, cudaMemcpyDeviceToHost, s),
                            "copy change");
                    launch_flip(e->g, d, m, s);
                    BB_CUDA(cudaGetLastError(), "sign flip");
                    bb_status st = wait_bounded(s, "incremental count");
                    if (st != BB_OK) return st;
                    const long long d3 = (long long)S.h->acc[1] - (long long)S.h->acc[2];
                    if (d3 % 3 != 0) return fail(BB_ERR_CUDA, "internal check failed (weighted change %lld)", d3);
                    e->last_balanced += d3 / 3;
                }
                t->balanced = e->last_balanced;
                t->total = e->last_total;
                t->incremental = true;
                return BB_OK;
            }
            launch_flip(e->g, d, m, s);
        } else {
            BB_CUDA(cudaMemcpyAsync(d, r.flip_idx, (size_t)r.n_flip * 8, cudaMemcpyHostToDevice, s),
                    "copy flip list");
            launch_flip(e->g, d, r.n_flip, s);
        }
        BB_CUDA(cudaGetLastError(), "sign flip");
    }
    e->have_counts = false;
    bb_status st = count_and_wait(S, e->g, t);
    if (st == BB_OK) {
        e->have_counts = true;
        e->last_balanced = t->balanced;
        e->last_total = t->total;
        e->g.h_wedges = S.h->wedges;  // the recount's cost, for the next flip decision
    }
    if (st != BB_OK && plan.fresh) plan.drop = true;
    return st;
}

void worker(Engine *E, int k) {
    cudaSetDevice(E->device);
    Slot &S = E->slots[k];
    std::unique_lock<std::mutex> lk(E->mu);
    for (;;) {
        bb_ticket_s *t = nullptr;
        Plan plan;
        while (!E->stop && !(t = pick(E, plan))) E->cv.wait(lk);
        if (!t) break;
        E->running++;
        lk.unlock();
        t->t_start = Clock::now();
        bb_status st = t->managed ? run_managed(E, S, t, plan) : count_and_wait(S, t->graph->g, t);
        if (st != BB_OK) t->err = bb_last_error();
        if (st == BB_ERR_TIMEOUT || st == BB_ERR_CUDA) plan.leak = true;
        lk.lock();
        if (plan.leak) {  // the device may still use these blocks: never hand them out again
            plan.temp.held = plan.flips.held = false;
            if (plan.entry) {
                plan.entry->graph.held = plan.entry->raw.held = false;
                plan.drop = true;
            }
        }
        release_block(E, plan.temp);
        release_block(E, plan.flips);
        if (t->managed) {
            Entry *e = plan.entry;
            e->busy = false;
            e->last_use = ++E->tick;
            if (plan.drop || (t->flags & BB_REQ_NO_CACHE)) remove_entry(E, e, false);
        } else {
            E->busy_graphs.erase(t->graph);
        }
        E->running--;
        t->st = st;
        if (st == BB_OK) E->stats.completed++; else E->stats.failed++;
        if (st == BB_OK && t->incremental) E->stats.incremental++;
        t->t_done = Clock::now();
        t->done.store(1, std::memory_order_release);
        E->cv.notify_all();
    }
}

void destroy_engine(Engine *E) {
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
        for (bb_ticket_s *t : E->queue) fail_now(E, t, BB_ERR_BUSY, "the serving engine stopped");
        E->queue.clear();
        E->cv.notify_all();
    }
    for (Slot &S : E->slots)
        if (S.th.joinable()) S.th.join();
    cudaSetDevice(E->device);
    for (Slot &S : E->slots) {
        // a slot's work still running after the wait limit keeps its stream
        if (S.s && wait_bounded(S.s, "serving slot") == BB_OK) cudaStreamDestroy(S.s);
        aux_destroy(S.aux);
        if (S.h) cudaFreeHost(S.h);
    }
    for (auto &kv : E->cache) delete kv.second;
    E->cache.clear();
    if (E->arena_mem) dev_free(E->ctx, E->arena_mem, E->arena_bytes);
    delete E;
}

// starts an engine (caller holds ctx->mu)
bb_status start_engine(bb_ctx *ctx, int slots, uint64_t arena_bytes) {
    Engine *E = new (std::nothrow) Engine();
    if (!E) return fail(BB_ERR_OOM, "host allocation failed");
    E->ctx = ctx;
    E->device = ctx->device;
    if (arena_bytes) {
        E->arena_bytes = Arena::round(arena_bytes);
        bb_status st = dev_alloc(ctx, (void **)&E->arena_mem, E->arena_bytes, "serving arena");
        if (st != BB_OK) { delete E; return st; }
        E->arena.reset(E->arena_bytes);
    }
    E->slots.resize(slots);
    for (Slot &S : E->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&S.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = aux_create(S.aux);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&S.h, sizeof(HostResult));
        if (e != cudaSuccess) {
            destroy_engine(E);
            return cuda_fail(e, "serving slot set-up");
        }
    }
    for (int k = 0; k < slots; k++) E->slots[k].th = std::thread(worker, E, k);
    ctx->engine = E;
    return BB_OK;
}

bb_status enqueue(bb_ctx *ctx, bb_ticket_s *t, bb_ticket *out) {
    Engine *E = ctx->engine;
    t->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(E->mu);
    if (E->stop) { delete t; return fail(BB_ERR_BUSY, "the serving engine is stopping"); }
    E->queue.push_back(t);
    E->stats.submitted++;
    *out = t;
    E->cv.notify_one();
    return BB_OK;
}

}  // namespace

void bb::engine_stop(bb_ctx *ctx) {
    if (!ctx || !ctx->engine) return;
    destroy_engine(ctx->engine);
    ctx->engine = nullptr;
}

extern "C" {

bb_status bb_ctx_serve(bb_ctx *ctx, int slots, uint64_t arena_bytes) {
    if (!ctx) return fail(BB_ERR_INVALID_ARG, "ctx is NULL");
    if (slots < 1 || slots > 64) return fail(BB_ERR_INVALID_ARG, "slots %d outside [1, 64]", slots);
    std::lock_guard<std::mutex> lk(ctx->mu);
    bb_status st = set_device(ctx);
    if (st != BB_OK) return st;
    if (ctx->engine) {  // drain, then replace
        Engine *E = ctx->engine;
        {
            std::unique_lock<std::mutex> elk(E->mu);
            E->cv.wait(elk, [&] { return E->queue.empty() && E->running == 0; });
        }
        engine_stop(ctx);
    }
    return start_engine(ctx, slots, arena_bytes);
}

bb_status bb_submit(bb_ctx *ctx, bb_graph *g, uint32_t flags, bb_ticket *out) {
    if (!ctx || !g || !out) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    if (flags) return fail(BB_ERR_INVALID_ARG, "flags must be 0");
    if (g->ctx != ctx) return fail(BB_ERR_INVALID_ARG, "graph belongs to another context");
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->engine) {
            bb_status st = set_device(ctx);
            if (st == BB_OK) st = start_engine(ctx, 2, 0);
            if (st != BB_OK) return st;
        }
    }
    bb_ticket_s *t = new (std::nothrow) bb_ticket_s();
    if (!t) return fail(BB_ERR_OOM, "host allocation failed");
    t->graph = g;
    return enqueue(ctx, t, out);
}

bb_status bb_submit_request(bb_ctx *ctx, const bb_request *req, uint32_t flags, bb_ticket *out) {
    if (!ctx || !req || !out) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    if (flags & ~BB_REQ_NO_CACHE) return fail(BB_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    if (req->n_flip < 0 || (req->n_flip > 0 && !req->flip_idx))
        return fail(BB_ERR_INVALID_ARG, "bad flip list");
    if (req->csr) {
        bb_status st = check_csr(req->csr, req->signs);
        if (st != BB_OK) return st;
    }
    if (!ctx->engine || ctx->engine->arena_bytes == 0)
        return fail(BB_ERR_INVALID_ARG,
                    "no managed cache: start the engine with bb_ctx_serve and arena_bytes > 0");
    bb_ticket_s *t = new (std::nothrow) bb_ticket_s();
    if (!t) return fail(BB_ERR_OOM, "host allocation failed");
    t->managed = true;
    t->req = *req;
    t->flags = flags;
    return enqueue(ctx, t, out);
}

bb_status bb_poll_timed(bb_ticket t, int *done, int64_t *balanced, int64_t *total,
                        double *queue_ms_opt, double *run_ms_opt) {
    if (!t || !done || !balanced || !total) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    if (!t->done.load(std::memory_order_acquire)) {
        *done = 0;
        return BB_OK;
    }
    *done = 1;
    using ms = std::chrono::duration<double, std::milli>;
    if (queue_ms_opt) *queue_ms_opt = ms(t->t_start - t->t_submit).count();
    if (run_ms_opt) *run_ms_opt = ms(t->t_done - t->t_start).count();
    const bb_status st = t->st;
    if (st == BB_OK) {
        *balanced = t->balanced;
        *total = t->total;
    } else {
        fail(st, "%s", t->err.c_str());
    }
    delete t;
    return st;
}

bb_status bb_poll(bb_ticket t, int *done, int64_t *balanced, int64_t *total) {
    return bb_poll_timed(t, done, balanced, total, nullptr, nullptr);
}

bb_status bb_ctx_serve_stats(bb_ctx *ctx, bb_serve_stats *out) {
    if (!ctx || !out) return fail(BB_ERR_INVALID_ARG, "NULL argument");
    *out = bb_serve_stats{};
    std::lock_guard<std::mutex> lk(ctx->mu);
    Engine *E = ctx->engine;
    if (!E) return BB_OK;
    std::lock_guard<std::mutex> elk(E->mu);
    *out = E->stats;
    out->resident_graphs = (int64_t)E->cache.size();
    out->arena_bytes = E->arena.capacity();
    out->arena_used = E->arena.used();
    out->arena_largest_free = E->arena.largest_free();
    out->queued = (int64_t)E->queue.size();
    out->running = E->running;
    return BB_OK;
}

}  // extern "C"
