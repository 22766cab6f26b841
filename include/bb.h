/*
 * bb.h - balanced butterfly counting on one GB300 GPU (sm_103a), C ABI.
 *
 * Problem (paper Section "Problem Definition", Defs. 1-2): a signed
 * bipartite graph G = (U, V, E) labels every edge + or -. A butterfly is a
 * 4-cycle u1 - v1 - u2 - v2; it is balanced when it has an even number of
 * negative edges. The library returns the number of balanced butterflies,
 * the number of all butterflies, and optionally, per vertex, the number of
 * balanced butterflies that contain it (Algorithm 3, Section "Extensions").
 *
 * Method (Section "Bucket Approach", Lemma 2 and Algorithm 2, made data
 * parallel as in Algorithm 4): vertices are ranked by degree priority
 * (Def. 4); the wedges u - v - w whose highest-priority vertex is an
 * endpoint are bucketed by endpoint pair and by wedge type (symmetric: both
 * edge signs equal, Def. 5; asymmetric: Def. 6); a pair with l symmetric and
 * m asymmetric wedges holds C(l,2) + C(m,2) balanced butterflies out of
 * C(l+m,2). All arithmetic is integer; results are exact.
 *
 * Input layout (every call that takes a graph):
 *   U-side CSR. rowptr: int64[nU+1], rowptr[0] = 0, non-decreasing,
 *   rowptr[nU] = nE. col: int32[nE], V ids in [0, nV); a row may be in any
 *   order but must not repeat a V id (E is a set). signs: int8[nE], each +1
 *   or -1, aligned with col.
 * Limits: nU + nV < 2^31, nE < 2^32 - 1 (so every degree and every
 *   per-pair wedge count is below 2^32). Counts per vertex pair are held in
 *   16-bit fields for anchors of degree <= 65535 and in 32-bit fields for
 *   the few of higher degree.
 *
 * Errors: every call returns a bb_status. On error no output is written and
 * bb_last_error() (thread-local) describes the failure. Device-side input
 * checks report BB_ERR_INVALID_ARG like host-side ones.
 *
 * Ownership: pointers passed in are borrowed for the duration of the call
 * unless stated otherwise. Objects created by the library (contexts, graphs)
 * are released by the matching destroy/free call.
 *
 * Threading: a context may be used from one thread at a time, except that
 * bb_poll may run concurrently with bb_submit.
 */
#ifndef BB_H
#define BB_H

#include <stdint.h>

#if defined(__GNUC__)
#define BB_API __attribute__((visibility("default")))
#else
#define BB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BB_OK = 0,
    BB_ERR_INVALID_ARG = 1, /* NULL pointer, bad CSR, sign not +-1, duplicate edge */
    BB_ERR_TOO_LARGE = 2,   /* beyond the limits above */
    BB_ERR_BUDGET = 3,      /* the call would exceed the context's device memory budget */
    BB_ERR_OOM = 4,         /* the device (or pinned host) allocation failed */
    BB_ERR_TIMEOUT = 5,     /* a bounded wait gave up */
    BB_ERR_OVERFLOW = 6,    /* a count does not fit in int64 */
    BB_ERR_CUDA = 7,        /* a CUDA runtime call failed */
    BB_ERR_NO_DEVICE = 8,   /* no usable CUDA device of compute capability 10.3 */
    BB_ERR_BUSY = 9         /* the serving engine stopped before running a request */
} bb_status;

typedef struct bb_ctx bb_ctx;
typedef struct bb_graph bb_graph;
typedef struct bb_ticket_s *bb_ticket;  /* an asynchronous request (bb_submit) */

/* U-side CSR of a signed bipartite graph (layout above). */
typedef struct {
    int64_t nU, nV, nE;
    const int64_t *rowptr;
    const int32_t *col;
} bb_csr;

/* Message for the last failing call on this thread ("" if none). */
BB_API const char *bb_last_error(void);

/* Library version string. */
BB_API const char *bb_version(void);

/* ---------------------------------------------------------------- context
 * A context binds one device, one CUDA stream and a device memory budget.
 * device: CUDA ordinal. hbm_budget_bytes: upper bound on device memory the
 * context may hold (0 = 90% of the device's free memory at creation). */
BB_API bb_status bb_ctx_create(int device, uint64_t hbm_budget_bytes, bb_ctx **out);
BB_API void bb_ctx_destroy(bb_ctx *ctx);

/* Run the context's work on `stream` (a cudaStream_t of the context's
 * device; NULL restores the context's own stream). */
BB_API bb_status bb_ctx_set_stream(bb_ctx *ctx, void *stream);

/* Device bytes the context holds now (graphs, workspaces). */
BB_API uint64_t bb_ctx_device_bytes(const bb_ctx *ctx);

/* ---------------------------------------------------------- one-shot count
 * The whole path on one graph: validate, degree-priority relabel,
 * sign-packed CSR build, work classification, wedge aggregation and the
 * C(.,2) reduction (Algorithm 2 and Lemma 2 over every wedge). Blocking.
 *
 * bb_count_csr: csr/signs in HOST memory (pinned memory makes the copies
 *   asynchronous); per_vertex_opt: NULL or host int64[nU+nV] (U ids, then V
 *   ids) receiving the balanced count of each vertex.
 * bb_count_csr_device: csr arrays, signs and per_vertex_opt in DEVICE
 *   memory of the context's device; the buffers are only read (written for
 *   per_vertex_opt) on the context's stream, during the call.
 * wedges_opt: NULL or receives the number of wedges aggregated.
 * The workspace grows to the largest graph seen and is reused. A call that
 * repeats the previous call's sizes and buffers (and timing setting)
 * replays the work after input validation from a CUDA graph captured at
 * the first repeat; the buffers' contents are read afresh by every call,
 * so results are those of the current inputs. The context's stream must
 * then be one that can be captured (not the legacy default stream, for
 * which every call launches directly). */
BB_API bb_status bb_count_csr(bb_ctx *ctx, const bb_csr *csr, const int8_t *signs, int64_t *balanced,
                       int64_t *total, int64_t *per_vertex_opt, int64_t *wedges_opt);
BB_API bb_status bb_count_csr_device(bb_ctx *ctx, const bb_csr *csr_dev, const int8_t *signs_dev,
                              int64_t *balanced, int64_t *total, int64_t *per_vertex_dev_opt,
                              int64_t *wedges_opt);

/* ------------------------------------------------------- resident graphs
 * bb_graph_upload: copies a host graph to the device, builds the ranked
 * sign-packed CSR and keeps it resident (counted against the budget).
 * bb_graph_upload_device: the same from device buffers (borrowed for the
 * call). */
BB_API bb_status bb_graph_upload(bb_ctx *ctx, const bb_csr *csr, const int8_t *signs, bb_graph **out);
BB_API bb_status bb_graph_upload_device(bb_ctx *ctx, const bb_csr *csr_dev, const int8_t *signs_dev,
                                 bb_graph **out);

/* Counts of a resident graph (wedge aggregation + reduction only). Blocking.
 * per_vertex_opt: NULL or host int64[nU+nV] as above. */
BB_API bb_status bb_count(bb_graph *g, int64_t *balanced, int64_t *total, int64_t *per_vertex_opt);

/* Balanced butterflies containing each edge of a resident graph (the
 * paper's edge-level extension of the per-vertex count, eBBFC; every
 * balanced butterfly adds one to each of its four edges, so the values sum
 * to 4 * balanced). per_edge: host int64[nE] in the input CSR's edge order.
 * balanced_opt / total_opt: NULL or the graph's counts. Blocking; device
 * workspace 24 bytes per edge (grow-only, within the context's budget). */
BB_API bb_status bb_count_edges(bb_graph *g, int64_t *per_edge, int64_t *balanced_opt,
                                int64_t *total_opt);

/* Flip the signs of the listed input edges (indices into the CSR's col
 * array; an index listed twice flips back) and return the graph's counts
 * after the flips. When the counts before the flips are known (the graph
 * was counted since its last plain bb_graph_flip_signs) and the butterflies
 * through the flipped edges are cheaper to enumerate than the whole graph's
 * wedges, only those are walked: a butterfly with an odd number of flipped
 * edges changes balance, the others do not (incremental re-count; the paper
 * has no counterpart beyond its edge-level extension). Otherwise the graph
 * is recounted, and always when its counts take the matrix-product path
 * (bb_set_matrix_product: such a recount costs less than any walk on a
 * graph that dense). *incremental_opt tells which was done. Blocking. */
BB_API bb_status bb_count_flipped(bb_graph *g, const int64_t *edge_idx, int64_t n,
                                  int64_t *balanced, int64_t *total, int *incremental_opt);

/* The same counts by the paper's baseline, BB-Base (Algorithm 1), on the
 * GPU: the middles of each vertex pair are grouped and every pair of them
 * is tested explicitly, so the work is the number of butterflies rather
 * than of wedges. Kept to measure the bucket method's advantage on the same
 * device; blocking; device workspace ~ (CTAs) x (largest anchor's wedges)
 * bytes. */
BB_API bb_status bb_count_base(bb_graph *g, int64_t *balanced, int64_t *total);

/* Negate the sign of the listed input edges (indices into the CSR's col
 * array, host int64[n]) in the resident graph, both directions. Repeated
 * indices flip repeatedly. Later counts see the new signs. */
BB_API bb_status bb_graph_flip_signs(bb_graph *g, const int64_t *edge_idx, int64_t n);

/* Graph facts: vertex and edge counts, wedges the count aggregates. */
/* Device bytes a graph of these sizes needs: `resident_opt` for as long as
 * it is kept (a bb_graph holds this plus its input copy, rowptr + col +
 * signs), `workspace_opt` during its build only. BB_ERR_INVALID_ARG on
 * negative sizes. */
BB_API bb_status bb_graph_bytes(int64_t nU, int64_t nV, int64_t nE, uint64_t *resident_opt,
                                uint64_t *workspace_opt);
BB_API bb_status bb_graph_info(const bb_graph *g, int64_t *nU, int64_t *nV, int64_t *nE,
                        int64_t *wedges);

BB_API void bb_graph_free(bb_graph *g);

/* ------------------------------------------------ allocation-free count
 * The paper has no counterpart to this call; it exists for callers that
 * cannot ask for device memory at the time they count: processes whose
 * device memory is already handed out by another allocator (a request would
 * fail or fragment it), and services that forbid allocation once they are
 * running (an allocation may block and synchronize the device).
 *
 * It runs the same path as bb_count_csr_device on csr_dev/signs_dev (device
 * memory of the current device) and writes the counts to host memory, but
 * needs no context and allocates nothing: every intermediate buffer is
 * carved out of one device array of BB_NOALLOC_SCRATCH_BYTES that the
 * library reserves on every GPU it is loaded on until the process exits.
 * A graph whose workspace does not fit is rejected with BB_ERR_TOO_LARGE
 * (roughly 1.3M edges of a power-law graph fit). Every call looks the
 * array's device address up on the current device; the first call on a
 * device may load the library's device code. Work is queued on `stream`
 * (NULL = the legacy default stream) and the call blocks until it is done
 * (it synchronizes with the stream); its waits honour bb_set_wait_timeout
 * (BB_ERR_TIMEOUT). All calls share the array and it keeps the last call's
 * contents: the call clears what must start at zero itself, and two calls
 * whose work overlaps on the GPU (another thread, another stream) race and
 * give wrong results. */
#define BB_NOALLOC_SCRATCH_BYTES (128u << 20)
BB_API bb_status bb_count_csr_device_noalloc(const bb_csr *csr_dev, const int8_t *signs_dev,
                                             void *stream, int64_t *balanced, int64_t *total,
                                             int64_t *wedges_opt);

/* ------------------------------------------------------------- tracing
 * Phase timings of the last count on a context, from CUDA events recorded
 * on the context's stream while timing is enabled (bb_ctx_set_timing).
 * Index 0/1/2/3 of the per-kernel arrays is the dense-counter, CTA-hash,
 * team and warp wedge kernel, in launch order; wedges/middles/anchors are
 * the work each kernel was given (middle = one neighbour v of an anchor w,
 * whose wedge suffix the kernel walks). build_ms covers validation through
 * classification (0 for resident-graph counts). product_ms is the time of
 * the matrix-product path (bb_set_matrix_product) when it counted instead
 * of the wedge kernels, whose entries are then 0; 0 otherwise. */
#define BB_NKERNELS 4
typedef struct {
    double build_ms;
    double count_ms;
    double kernel_ms[BB_NKERNELS];
    int64_t wedges[BB_NKERNELS];
    int64_t middles[BB_NKERNELS];
    int64_t anchors[BB_NKERNELS];
    double product_ms;
} bb_timing;

BB_API bb_status bb_ctx_set_timing(bb_ctx *ctx, int enable);
BB_API bb_status bb_ctx_last_timing(const bb_ctx *ctx, bb_timing *out);

/* ------------------------------------------------------ bucket shapes
 * The work classes of a graph's anchors (Algorithm 2's per-start work,
 * bucketed by wedge count and endpoint range; this library's division of
 * the paper's bucket loop into kernels) have runtime bounds, none of which
 * changes a count:
 *   warp_w_max:   warp-class anchors have at most this many wedges
 *                 (1..16384, default 16384; degree <= 255 is fixed);
 *   warp_small_w: warp-class anchors with at most this many wedges keep
 *                 every endpoint in a hash instead of the hub window
 *                 (0..warp_w_max, default 32);
 *   team_w_max:   team-class anchors have at most this many wedges
 *                 (1..16384, default 16384);
 *   split_wedges: a dense anchor is split over CTAs into parts of at least
 *                 this many wedges (1024..2^30, default 65536).
 * dense_staged (0/1, default 0): the dense-class walker stages the
 * middles' rows in shared memory by bulk copies instead of loading them
 * directly.
 * bb_ctx_set_shape: used by the context's later one-shot counts and
 *   uploads (shape NULL = the defaults). BB_ERR_INVALID_ARG outside the
 *   ranges above.
 * bb_graph_set_shape: re-classifies a resident graph (its rows are kept;
 *   blocking; uses the context's build workspace). */
typedef struct {
    uint32_t warp_w_max;
    uint32_t warp_small_w;
    uint32_t team_w_max;
    uint32_t split_wedges;
} bb_class_shape;

BB_API bb_status bb_ctx_set_shape(bb_ctx *ctx, const bb_class_shape *shape, int dense_staged);
BB_API bb_status bb_graph_set_shape(bb_graph *g, const bb_class_shape *shape, int dense_staged);

/* ------------------------------------------------------------- batches
 * Many resident graphs counted together: every graph's wedge work goes
 * into one shared work queue per work class (dense-counter, CTA-hash, team
 * and warp anchors; the classes come from each anchor's wedge count and
 * endpoint range, Algorithm 2's per-start work), and one persistent kernel
 * per class drains its queue across all graphs. The whole sequence (reset,
 * four class kernels, result gather and copy-back) is captured once as a
 * CUDA graph and replayed by each bb_batch_count. Each graph's counts are
 * exactly what bb_count gives for it alone. The paper counts one graph at
 * a time; batching is this library's addition.
 *
 * bb_batch_create: `graphs` (host array of n resident graphs of one context)
 *   is copied; the graphs must outlive the batch and must not be freed
 *   while it exists. Sign flips of member graphs are seen by later counts.
 *   Device memory: ~n*600 bytes plus 40 bytes per graph of results, within
 *   the context's budget (BB_ERR_BUDGET otherwise).
 * bb_batch_count: blocking. balanced/total: host int64[n]; status_opt: NULL
 *   or host bb_status[n]. A graph whose count fails gets -1 in both outputs
 *   and its status; the call then returns the first such status (message
 *   names the graph index). The first call captures the CUDA graph on the
 *   context's stream, which must not be the legacy default stream. With
 *   timing enabled on the context (bb_ctx_set_timing) the count runs
 *   uncaptured, classes one after another, and bb_ctx_last_timing gives
 *   each class kernel's time and work (wedges, middles, anchors) summed
 *   over the members.
 * bb_batch_tune: launch shapes per work class, index order as in bb_timing
 *   (dense, CTA-hash, team, warp). warp_chunk: warp anchors a warp takes
 *   per grab (1..1024); concurrent: 1 = the class kernels run on separate
 *   streams at once, 0 = one after another; grid_frac: each class kernel's
 *   grid as a fraction (0, 1] of its full-occupancy grid; dense_staged: as
 *   above, for the whole batch. shape[k]: the bucket shape of the members
 *   in size class k (fewer than 2^14, 2^17, 2^20 edges, and the rest); a
 *   changed shape re-classifies that class's members (blocking).
 * bb_batch_autotune: times candidate shapes on this batch (each `reps`
 *   times, median) by coordinate descent over the launch shapes and each
 *   size class's bucket shape, keeps the fastest (also written to
 *   best_opt) and its time (best_ms_opt). Runs the counts it times. */
#define BB_NSIZE 4
typedef struct bb_batch bb_batch;
typedef struct {
    uint32_t warp_chunk;
    uint32_t concurrent;
    float grid_frac[BB_NKERNELS];
    uint32_t dense_staged;
    bb_class_shape shape[BB_NSIZE];
} bb_batch_tune;

BB_API bb_status bb_batch_create(bb_ctx *ctx, bb_graph *const *graphs, int64_t n, bb_batch **out);
BB_API bb_status bb_batch_count(bb_batch *b, int64_t *balanced, int64_t *total,
                                bb_status *status_opt);
BB_API bb_status bb_batch_set_tune(bb_batch *b, const bb_batch_tune *tune);
BB_API bb_status bb_batch_get_tune(const bb_batch *b, bb_batch_tune *out);
BB_API bb_status bb_batch_autotune(bb_batch *b, int reps, bb_batch_tune *best_opt,
                                   double *best_ms_opt);
BB_API void bb_batch_free(bb_batch *b);

/* ------------------------------------------------------------- serving
 * Asynchronous counts for a request loop. A context's serving engine runs
 * `slots` worker slots, each with its own CUDA stream: requests are queued
 * in arrival order and admitted as soon as a slot is free and their device
 * memory fits, so the uploads, builds and counts of several requests
 * overlap on the device (continuous batching: admission never waits for a
 * whole batch to finish). Two requests on the same graph run one after the
 * other. A request's counts are exactly what bb_count gives for the graph.
 * The paper counts one graph per call; the serving engine is this
 * library's addition.
 *
 * bb_ctx_serve: starts (or restarts, after draining) the engine. arena_bytes
 *   is reserved at once from the context's budget and holds every graph of
 *   the managed cache with its input copy and build workspace (0 = no
 *   managed cache: only bb_submit of caller-owned graphs). Optional: the
 *   first bb_submit starts an engine with 2 slots and no cache.
 * bb_submit: count of a resident graph the caller owns (bb_graph_upload);
 *   the graph must not be freed, counted, flipped or batched until the
 *   ticket is done. flags must be 0.
 * bb_submit_request: count of the graph the caller names by `key`. A key
 *   not in the cache is uploaded from csr/signs (host pointers, borrowed
 *   until the ticket is done) into the arena, evicting the least recently
 *   used idle graphs as needed; a key in the cache is counted in place,
 *   after flipping the signs of the listed input edges (host int64
 *   indices, borrowed likewise; the flips stay); a small flip set on a graph
 *   whose counts are known is re-counted through the flipped edges only,
 *   as in bb_count_flipped. csr may be NULL when the
 *   caller knows the key is resident (the request fails with
 *   BB_ERR_INVALID_ARG if it is not). A graph larger than the arena fails
 *   with BB_ERR_BUDGET. flags: 0, or BB_REQ_NO_CACHE to drop the graph
 *   from the cache once counted.
 * bb_poll: never blocks. *done = 1 when the request has finished; then the
 *   return value is its status, balanced/total are written on success, and
 *   the ticket is released (it must not be used again). *done = 0: BB_OK,
 *   nothing else written. bb_poll_timed adds the milliseconds from submit
 *   to admission (queue_ms_opt) and from admission to completion
 *   (run_ms_opt), from the library's steady clock.
 * Threading: submit from one thread, poll from one (possibly the same).
 * bb_ctx_destroy waits for running requests; queued ones finish with
 * BB_ERR_BUSY and still need a bb_poll to be released. */
typedef struct {
    uint64_t key;
    const bb_csr *csr;
    const int8_t *signs;
    const int64_t *flip_idx;
    int64_t n_flip;
} bb_request;

#define BB_REQ_NO_CACHE 1u

typedef struct {
    int64_t submitted, completed, failed;
    int64_t cache_hits, uploads, evictions;
    int64_t resident_graphs;
    uint64_t arena_bytes, arena_used, arena_largest_free;
    int64_t queued, running;
    int64_t incremental;   /* re-queries counted through their flipped edges only */
} bb_serve_stats;

BB_API bb_status bb_ctx_serve(bb_ctx *ctx, int slots, uint64_t arena_bytes);
BB_API bb_status bb_submit(bb_ctx *ctx, bb_graph *g, uint32_t flags, bb_ticket *out);
BB_API bb_status bb_submit_request(bb_ctx *ctx, const bb_request *req, uint32_t flags,
                                   bb_ticket *out);
BB_API bb_status bb_poll(bb_ticket t, int *done, int64_t *balanced, int64_t *total);
BB_API bb_status bb_poll_timed(bb_ticket t, int *done, int64_t *balanced, int64_t *total,
                               double *queue_ms_opt, double *run_ms_opt);
BB_API bb_status bb_ctx_serve_stats(bb_ctx *ctx, bb_serve_stats *out);

/* Process-wide limit, in seconds, on how long a blocking call waits for its
 * device work (default 600). When it runs out the call returns
 * BB_ERR_TIMEOUT and its outputs are untouched; the work it queued still
 * runs, and later calls on the same context's stream run after it (their
 * waits, including the input validation, honour the same limit). The
 * release calls (bb_ctx_destroy, bb_graph_free, bb_batch_free) wait for the
 * object's queued work within the limit too; when it runs out they return
 * without freeing the object's device memory (it stays allocated, rather
 * than being freed under running work).
 * BB_ERR_INVALID_ARG unless 0 < seconds <= 86400. */
BB_API bb_status bb_set_wait_timeout(double seconds);

/* Failure injection for tests (no paper counterpart): the nth device
 * allocation the library makes from now on (workspaces, resident graphs,
 * batches, the serving arena; nth >= 1) fails once with BB_ERR_OOM as if
 * cudaMalloc had failed, so that callers can check how they recover.
 * 0 disarms it; BB_ERR_INVALID_ARG for nth < 0. Process-wide. */
BB_API bb_status bb_set_alloc_failure(int64_t nth);

/* Measurement probe: shared-memory atomic adds per second on `device`, each
 * a u32 atomicAdd whose previous value is used (the wedge kernels' inner
 * step) on a pseudo-random counter of a `window`-entry array (32..49152),
 * the whole GPU busy. The best of three timed runs after a warm-up. The
 * paper has no counterpart; it gives the count kernels' second ceiling. */
BB_API bb_status bb_probe_shared_atomics(int device, uint32_t window, double *atomics_per_s);

/* Kernel launches the library has issued in this process. */
BB_API uint64_t bb_launch_count(void);

/* ------------------------------------------------- matrix-product path
 * Lemma 2 per pair of vertices on one side, with the pair's symmetric and
 * asymmetric tallies (Defs. 5-6) taken over all middles at once: for the
 * a x b signed adjacency X of the smaller side (rows) against the other
 * (columns), X X^T holds S - A and |X| |X|^T holds S + A per pair, and the
 * counts are the sums of C(S,2) + C(A,2) and C(S+A,2) over the pairs. The
 * paper enumerates wedges instead; on a graph whose smaller side is small
 * and dense the two products (tensor-core GEMMs in bf16 with fp32 sums,
 * exact for these integer operands) take less time than the wedges.
 * Counts through bb_count_csr, bb_count_csr_device, resident graphs and
 * the serving engine take this path when the graph qualifies: the smaller
 * side has 2..8192 vertices, the other fewer than 2^21, there are at least
 * 65,536 edges and at least one edge per 16 vertex pairs across the sides
 * (and the two bf16 matrices fit 512 MiB each); the graph's device
 * workspace then includes the matrices (bb_graph_bytes). Per-vertex and
 * per-edge counts, flips, batches, BB-Base and the allocation-free call
 * always use the wedge path. Results are identical on both paths.
 * bb_set_matrix_product: process-wide, 0 = take the path when the graph
 * qualifies (default), 1 = always the wedge kernels; returns the previous
 * mode (-1 for another value). A count whose step was captured for replay
 * under the other mode is captured again.
 * bb_matrix_product_plan: 1 if a graph of these sizes would be counted on
 * this path under the current mode, 0 if not, -1 for a negative size. */
BB_API int bb_set_matrix_product(int mode);
BB_API int bb_matrix_product_plan(int64_t nU, int64_t nV, int64_t nE);

#ifdef __cplusplus
}
#endif

#endif /* BB_H */
