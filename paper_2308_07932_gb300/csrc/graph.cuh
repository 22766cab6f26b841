// graph.cuh - device-resident graph built for counting, and the work
// classes of its anchors.
//
// Wedges and anchors. Algorithm 2 counts, for every wedge u - v - w in which
// u has the highest priority of the three (Def. 4), one symmetric or
// asymmetric tally for the pair (u, w). Those tallies are kept here at the
// LOWER-priority endpoint w (the "anchor") keyed by the higher one u: the
// wedge set and every pair's (symmetric, asymmetric) counts are exactly
// Algorithm 2's, only the place where a pair's counters live differs. For an
// anchor w the wedges are w - v - u for every neighbour v of w and every u in
// the suffix of v's row ranked above both v and w; their endpoints u are the
// same-side vertices ranked above w, so an anchor never needs more counters
// than there are vertices above it on its side.
#pragma once
#include <cstdint>
#include "../../include/bb.h"
#include "common.cuh"

namespace bb {

// Hub window: the top HUB_WINDOW side ranks of the anchor's side. Wedge
// endpoints concentrate on these high-degree vertices, so team kernels keep
// them in dense counters and hash only the rest.
constexpr uint32_t HUB_WINDOW = 2048;
// dense counters per CTA job: 16Ki u32 (64 KiB of shared memory), so that
// three 512-thread dense CTAs share an SM (one 1024-thread CTA with 48Ki
// counters per SM was 35 % slower on the 2M x 500k graph)
constexpr uint32_t DENSE_CAP = 16384;
// warp class: one warp per anchor of degree <= WARP_DEG_MAX (its per-pair
// counts then fit 8 bits) and at most WARP_W_MAX wedges. Anchors with at
// most WARP_SMALL_W wedges hash every endpoint; larger ones keep the hub
// window in 16-bit counters and hash the rest; the hash has WARP_CAP slots.
constexpr uint32_t WARP_DEG_MAX = 255;
constexpr uint64_t WARP_W_MAX = 16384;
constexpr uint64_t WARP_SMALL_W = 32;
constexpr uint32_t WARP_CAP = 256;
// team class (4 warps): wedges <= TEAM_W_MAX, below-window wedges that fit
// a TEAM_CAP-slot hash, and at most TEAM_DEG_MAX middles (a team scans its
// middles 128 at a time; an anchor of many middles with few wedges, such as
// a high-degree vertex whose neighbours rank above it, goes to a 512-thread
// class instead: one such anchor of 20,261 middles took 0.26 ms as a team)
constexpr uint64_t TEAM_W_MAX = 16384;
constexpr uint32_t TEAM_CAP = 1024;
constexpr uint32_t TEAM_DEG_MAX = 2048;
// CTA hash class: below-window wedges that fit a CTAH_CAP-slot hash (64 KiB:
// two or three CTAs per SM; 16Ki slots held one and was 75 % slower)
constexpr uint32_t CTAH_CAP = 8192;
// split one dense anchor over several CTAs when its wedges exceed both this
// and 4x its endpoint range; parts are merged before the C(.,2) step
constexpr uint64_t SPLIT_WEDGES = 65536;
constexpr uint32_t MAX_PARTS = 64;
constexpr uint32_t MAX_SPLIT_JOBS = 1u << 16;
constexpr uint32_t MAX_GPART = 1u << 24;

enum Cls : uint32_t { CLS_WARP = 0, CLS_TEAM = 1, CLS_CTAH = 2, CLS_DENSE = 3, NCLS = 4 };

// The bucket shape of a graph's classification (runtime values within the
// compile-time bounds above): warp-class anchors have at most warp_w_max
// wedges and those with at most warp_small_w hash every endpoint; team
// anchors have at most team_w_max wedges; dense anchors are split into
// parts of at least split_wedges wedges.
struct ClassifyParams {
    uint32_t warp_w_max = (uint32_t)WARP_W_MAX;
    uint32_t warp_small_w = (uint32_t)WARP_SMALL_W;
    uint32_t team_w_max = (uint32_t)TEAM_W_MAX;
    uint32_t split_wedges = (uint32_t)SPLIT_WEDGES;
};

// One anchor in a class list: (side rank << 1 | side), start of its row,
// degree, wedges and below-window wedges (saturated to 32 bits), flags
// (bit 0: a warp-class anchor that hashes every endpoint).
constexpr uint32_t REC_HASH_ALL = 1u;
struct alignas(16) AnchorRec {
    uint32_t anchor, rb, deg, W;
    uint32_t wnh, flags, pad1, pad2;
};

// One CTA job over dense counters: anchor (side rank << 1 | side), its
// middle slice [m0, m1) of the anchor's row, and the split group (or
// NO_GROUP). A job whose anchor has more than DENSE_CAP vertices above it
// walks the endpoint range in DENSE_CAP windows.
constexpr uint32_t NO_GROUP = 0xffffffffu;
// group of a wide job: an anchor of degree above MAX_DEGREE, walked whole
// by one CTA with 32-bit tally fields (never split)
constexpr uint32_t WIDE_JOB = 0xfffffffeu;
struct DenseJob {
    uint32_t anchor;
    uint32_t m0, m1;
    uint32_t group;
};

struct SplitGroup {
    uint32_t parts;   // CTAs contributing partial counters
    uint32_t goff;    // offset of the merged counters in the partial buffer
    uint32_t len;     // counters (endpoint range length)
    uint32_t pad;
};

// counters written by the classifier
enum Ctr : uint32_t {
    CTR_WARP = 0, CTR_TEAM = 1, CTR_CTAH = 2, CTR_DENSE = 3, CTR_GROUPS = 4, CTR_GPART = 5,
    CTR_SPLITJOBS = 6, CTR_MAXDEG = 7, NCTR = 8
};

// per-count scratch (zeroed before each count)
struct CountScratch {
    unsigned long long acc[4];   // balanced lo/hi, total lo/hi (128-bit sums)
    unsigned long long cells;    // matrix-product path: distinct nonzero cells of X
    uint32_t job_next[7];        // dynamic job cursors: one per class, the split parts'
                                 // second walks, the per-vertex baseline, the wide jobs
    uint32_t err;
    uint32_t pad[1];
};
constexpr int JOB_PV_SPLIT = 4;
constexpr int JOB_BASE = 5;
constexpr int JOB_WIDE = 6;

// ------------------------------------------------------ matrix-product path
// On a graph with a small, dense side the tallies of every pair on that
// side over all middles come from two dense products of its a x b signed
// adjacency X (entries +1, -1, 0; rows the pair side P, columns the other
// side): X X^T holds S - A and |X| |X|^T holds S + A for each pair (Defs.
// 5-6), so the count is the sum over pairs of C(S,2) + C(A,2) and
// C(S+A,2) (Lemma 2) without enumerating wedges. Each butterfly has exactly
// one pair of P vertices, so no priority order is needed on this path.
// The products run on the tensor cores in bf16 with fp32 sums: every
// product is exactly -1, 0 or 1 and every partial sum an integer of
// magnitude at most b < 2^21, so the sums are exact.
//
// product_plan picks the path from the sizes alone (the same answer for a
// graph's workspace sizing, layout and launch): the smaller side as P, at
// most PROD_A_MAX pair vertices, fewer than PROD_B_MAX middles, at least
// PROD_MIN_EDGES edges, and an edge density of at least 1/PROD_DENSITY
// (where the products' a^2 b work is below the wedges' b (nE/b)^2 / 2 at
// the measured rates of both). side = -1: the wedge classes count.
constexpr uint32_t PROD_A_MAX = 8192;
constexpr uint32_t PROD_B_MAX = 1u << 21;
constexpr int64_t PROD_MIN_EDGES = 1 << 16;
constexpr int64_t PROD_DENSITY = 16;
constexpr uint64_t PROD_MAX_CELLS = 1ull << 28;  // a * ld: 512 MiB per bf16 matrix
// The middles are split into `split` equal slices of kc columns and each
// product is a batch of one GEMM per slice (partial a x a sums, added by
// the pair kernel in integers), so that a small pair side still gives the
// GPU about PROD_TARGET_TILES output tiles of 128 x 128 to work on.
constexpr uint32_t PROD_TARGET_TILES = 1024;
constexpr uint32_t PROD_MIN_SLICE = 1024;
struct ProductPlan {
    int side = -1;          // pair side (0 = U, 1 = V), -1 = wedge classes
    uint32_t a = 0, b = 0;  // pair-side and middle-side vertex counts
    uint32_t ap = 0;        // rows of X: a rounded up to 16 (the rest zero)
    uint32_t split = 1;     // middle slices (GEMMs per product)
    uint32_t kc = 0;        // columns per slice (a multiple of 64: 128-byte slices)
    uint32_t ld = 0;        // row pitch of X in elements: split * kc >= b
    size_t x_bytes = 0;     // X then |X| (bf16, ap x ld each)
    size_t c_bytes = 0;     // per product and slice an ap x ap fp32 partial
    size_t cnt_bytes = 0;   // wedge count: global ranks by id (a + b), and
                            // per row and column its cells and cells ranked above
    size_t ws_bytes = 0;    // GEMM workspace
    size_t total = 0;       // device bytes of all, 256-byte aligned
};
ProductPlan product_plan(int64_t nU, int64_t nV, int64_t nE);

// Process-wide choice between the paths for graphs the plan admits (0 =
// product when planned, 1 = always the wedge classes); see
// bb_set_matrix_product.
bool product_enabled();

struct DevGraph {
    int64_t nU = 0, nV = 0, nE = 0;
    SideCSR side[2];
    // raw input kept for flips (device; may be null for one-shot builds)
    int64_t *rowptr = nullptr;
    int32_t *col = nullptr;
    int8_t *sign = nullptr;
    // classification
    AnchorRec *warp_list = nullptr;
    AnchorRec *team_list = nullptr;
    AnchorRec *ctah_list = nullptr;
    DenseJob *dense_jobs = nullptr;
    SplitGroup *groups = nullptr;
    uint32_t *gpart = nullptr;       // merged partial counters of split anchors
    uint32_t gpart_cap = 0;          // entries in gpart
    uint32_t *gdone = nullptr;       // per group arrival counters
    uint32_t *ctr = nullptr;         // [NCTR]
    unsigned long long *wedges = nullptr;  // [1]
    // per work class (warp, team, CTA-hash, dense): wedges, middle steps, anchors
    unsigned long long *cls_stats = nullptr;  // [3 * NCLS]
    uint32_t *err = nullptr;         // build error word
    CountScratch *scratch = nullptr;
    // host copies after the build
    uint32_t h_ctr[NCTR] = {};
    uint64_t h_wedges = 0;
    ClassifyParams cls;      // bucket shape the classes were (or are to be) built with
    bool dense_staged = false;  // dense walker: rows staged by bulk copies (launch choice)
    uint32_t h_maxdeg = 0;   // largest vertex degree (read back by build_validate)
    int deg_bits = 16;       // key bits of the degree sort (16, 24 or 32, from h_maxdeg)
    unsigned long long h_cls_stats[3 * NCLS] = {};  // resident graphs: copy of cls_stats
    // matrix-product path (prod.side >= 0 when the layout reserved it);
    // product_only: built for that path alone (ranks and the wedge count;
    // no rows, descriptors or classes), so only it may count the graph
    ProductPlan prod;
    bool product_only = false;
    uint16_t *prod_x = nullptr;  // [2][ap][ld] bf16 bit patterns: X, |X|
    float *prod_c = nullptr;     // [2][split][ap][ap]: partials of X X^T, |X| |X|^T
    uint32_t *prod_cnt = nullptr;  // [a + b] ranks, [2][ap] row and [2][ld] column counts
    void *prod_ws = nullptr;     // GEMM workspace (prod.ws_bytes)
};

// Bytes of device memory a graph of this size needs (graph + build temps).
struct BuildSizes {
    size_t graph_bytes;   // kept while the graph lives
    size_t temp_bytes;    // needed only during the build
};
// product = false: no matrix-product buffers (the graph always takes the
// wedge classes); layout_graph must be given the same choice.
BuildSizes build_sizes(int64_t nU, int64_t nV, int64_t nE, bool product = true);

// Carve the graph's arrays out of `graph_mem` (graph_bytes long).
void layout_graph(DevGraph &g, int64_t nU, int64_t nV, int64_t nE, void *graph_mem,
                  bool product = true);

// Two auxiliary streams and their events the build may fork work onto (both
// are joined back to s before the build's later stages): the long-row radix
// sorts run on `stream`, the V side's shorter-row sorts on `stream2`.
struct BuildAux {
    cudaStream_t stream = nullptr, stream2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
};
cudaError_t aux_create(BuildAux &a);   // non-blocking streams, timing-free events
void aux_destroy(BuildAux &a);         // waits (bounded) for both streams; safe on a partial create

// Waits for the work queued so far on s (BB_ERR_TIMEOUT after the
// library's wait limit, bb_set_wait_timeout). wait_stream_bounded waits
// until s is idle instead and creates no CUDA object (for paths that must
// not).
bb_status wait_bounded(cudaStream_t s, const char *what);
bb_status wait_stream_bounded(cudaStream_t s, const char *what);

// Build from device CSR (rowptr/col/sign on the device). Sets *verr to 0 or
// the input-check error bits; returns BB_OK, or the failure of the one wait
// (on the validation check). aux may be null (all work on s). The two
// stages separately: build_validate (resets, input checks and degrees;
// waits for the check, bounded, and reads back its error bits and the
// largest degree) and build_rest (everything after, no host
// synchronisation: it can be captured in a CUDA graph).
bb_status build_graph(DevGraph &g, const int64_t *rowptr, const int32_t *col, const int8_t *sign,
                      void *temp_mem, cudaStream_t s, const BuildAux *aux, uint32_t *verr);
// Inputs still arriving (host-to-device copies on another stream): the
// validation waits on each part's event before checking it, so the checks
// of early edge chunks overlap the copies of later ones.
struct StagedInput {
    static constexpr int MAX_CHUNKS = 8;
    int chunks = 0;                         // edge chunks
    int64_t lo[MAX_CHUNKS + 1] = {};        // chunk c: edges [lo[c], lo[c+1])
    cudaEvent_t rowptr_ready = nullptr;
    cudaEvent_t ready[MAX_CHUNKS] = {};
};
// pin_err / pin_max: optional pinned host words that receive the error
// word and the largest degree behind the checks (saves two pageable copies
// after the wait).
bb_status build_validate(DevGraph &g, const int64_t *rowptr, const int32_t *col, const int8_t *sign,
                         void *temp_mem, cudaStream_t s, const StagedInput *in, uint32_t *verr,
                         uint32_t *pin_err = nullptr, uint32_t *pin_max = nullptr);
// product_only: stop after the ranks (a graph that the matrix-product
// path counts next, on the same inputs, and whose wedges that path counts;
// sets g.product_only).
void build_rest(DevGraph &g, const int64_t *rowptr, const int32_t *col, const int8_t *sign,
                void *temp_mem, cudaStream_t s, const BuildAux *aux, bool product_only = false);

// Re-runs the classification of a built graph with g.cls (the class lists,
// dense jobs and split groups are rewritten; the rows, descriptors and
// work counts are kept). ctemp: device scratch of classify_temp_bytes.
// Asynchronous on s; the host copies (h_ctr, h_cls_stats) are stale until
// the caller reads ctr and cls_stats back.
size_t classify_temp_bytes(int64_t nU, int64_t nV);
void classify_graph(DevGraph &g, void *ctemp, cudaStream_t s);

// Count balanced/total butterflies of a built graph on stream s. Writes the
// 128-bit sums to g.scratch->acc (device). When ev is not null, ev[0..4]
// are recorded before the dense, CTA-hash, team and warp kernels and after
// the last one. Returns true when the matrix-product path counted instead
// (then ev[0] precedes it and ev[1..4] follow it).
bool launch_count(const DevGraph &g, cudaStream_t s, cudaEvent_t *ev = nullptr);

// The matrix-product path on stream s (g.prod.side >= 0): adds the sums to
// g.scratch->acc. Returns false, with nothing counted, when the GEMM library
// could not be set up or refused the call (the caller counts with the
// wedge classes then).
bool launch_product(const DevGraph &g, cudaStream_t s);

// Sets up the GEMM library on the current device (once); false if it
// cannot be used (then no graph is built for the product path alone).
bool product_ready();

// Many resident graphs counted in one launch per work class. Items of class
// c of graph i are numbered prefix[c*(n+1)+i] .. prefix[c*(n+1)+i+1]-1 in
// one space (prefix built from each graph's class counters). After the
// launch, out[i*BATCH_OUT ..] holds graph i's 128-bit balanced and total
// sums and its error words (count | build << 32).
constexpr int BATCH_OUT = 5;
struct BatchLaunch {
    const DevGraph *graphs;   // device [n]
    const uint32_t *prefix;   // device [NCLS * (n + 1)]
    uint32_t *next;           // device [NCLS]
    unsigned long long *out;  // device [n * BATCH_OUT]
    uint32_t n;
    uint32_t items[NCLS];     // host copy of the prefix totals
};
// Launch shapes: items a warp takes per grab, whether the classes run on
// separate streams at once, and each class's grid as a fraction of its
// full-occupancy grid.
// Bucket shapes per graph-size class of a batch: members with fewer than
// 2^14, 2^17, 2^20 edges, and the rest.
constexpr int NSIZE = 4;
inline int size_class(int64_t nE) {
    return nE < (1 << 14) ? 0 : nE < (1 << 17) ? 1 : nE < (1 << 20) ? 2 : 3;
}
struct BatchTune {
    uint32_t warp_chunk = 8;
    uint32_t concurrent = 1;
    float grid_frac[NCLS] = {1.f, 1.f, 1.f, 1.f};
    uint32_t dense_staged = 0;
    ClassifyParams shape[NSIZE];
};
// side: NCLS-1 streams and ev: NCLS events, used when T.concurrent is set
// (both may be null otherwise). Works under stream capture. tev (optional,
// NCLS+1 timing events) turns concurrency off and brackets the class
// kernels in the order dense, CTA-hash, team, warp.
void launch_count_batch(const BatchLaunch &L, const BatchTune &T, cudaStream_t s,
                        const cudaStream_t *side, const cudaEvent_t *ev,
                        const cudaEvent_t *tev = nullptr);
int batch_max_blocks(int cls);
// gathers every member's class counters (NCTR per graph) and class
// statistics (3 * NCLS per graph) into device arrays
void launch_batch_classes(const BatchLaunch &L, uint32_t *ctr_dev, unsigned long long *stats_dev,
                          cudaStream_t s);

// The count of launch_count (same sums, same events) together with the
// balanced butterflies containing each vertex (Algorithm 3's quantity) of
// a built graph: written to out_dev (device int64[nU+nV], U ids then V ids).
void launch_per_vertex(const DevGraph &g, int64_t *out_dev, cudaStream_t s,
                       cudaEvent_t *ev = nullptr);

// The count together with the balanced butterflies containing each input
// edge of a built graph that keeps its raw input (rowptr/col): written to
// out_dev (device int64[nE], input CSR order); pe_ws is device scratch of
// 2 * nE u64.
void launch_per_edge(const DevGraph &g, int64_t *out_dev, unsigned long long *pe_ws,
                     cudaStream_t s, cudaEvent_t *ev = nullptr);

// Incremental re-count under sign flips (flips.cu). The workspace of
// flip_ws_bytes(nE, n) holds the located edges and two flag bitmaps.
// launch_flip_estimate locates the n listed input edges (distinct), marks
// them and writes the enumeration cost to cost_dev; launch_flip_delta then
// writes the weighted changes to acc_dev[0] (up) and acc_dev[1] (down):
// the balanced count changes by (up - down) / 3. Both read the signs
// before the flips are applied (launch_flip afterwards).
size_t flip_ws_bytes(int64_t nE, int64_t n);
void launch_flip_estimate(const DevGraph &g, const int64_t *edges_dev, int64_t n, void *ws,
                          unsigned long long *cost_dev, cudaStream_t s);
void launch_flip_delta(const DevGraph &g, int64_t n, void *ws, unsigned long long *acc_dev,
                       cudaStream_t s);

// BB-Base (Algorithm 1) for comparison (base.cu): explicit pair tests.
// launch_max_work writes the largest anchor wedge count to out_dev;
// launch_base needs base_blocks() per-CTA buffers of that many bytes and
// writes balanced / total to acc_dev[0] / acc_dev[1].
int base_blocks();
void launch_max_work(const DevGraph &g, unsigned long long *out_dev, cudaStream_t s);
void launch_base(const DevGraph &g, uint8_t *scratch, uint64_t per_cta,
                 unsigned long long *acc_dev, cudaStream_t s);

// Flip the signs of listed input edges (device list of n indices).
void launch_flip(DevGraph &g, const int64_t *edge_idx_dev, int64_t n, cudaStream_t s);

// One-time per-device kernel attributes (shared-memory opt-ins, grids).
void count_init();

// Records a timing event on s; while s is being captured into a CUDA graph
// the record is made an external one (an event record node that fires at
// each replay, not a dependency inside the capture).
inline void record_timing_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

// Sets the calling thread's bb_last_error() message; returns st.
bb_status report_error(bb_status st, const char *msg);

// entries of the split-merge buffer for a graph with nE edges
inline size_t gpart_entries(int64_t nE) {
    size_t want = (size_t)4 * (size_t)nE + 4096;
    return want < MAX_GPART ? want : MAX_GPART;
}

}  // namespace bb
