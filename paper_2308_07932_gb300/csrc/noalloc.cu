// noalloc.cu - bb_count_csr_device_noalloc: the whole count of a graph
// already on the device, with every intermediate buffer carved out of one
// file-scope device array instead of allocated memory.
//
// The array is reserved in every GPU that loads the library, for the life of
// the process. Host code cannot use the array's name as a device address, so
// every call looks the address up (cudaGetSymbolAddress, with the caller's
// device current; cheap once the library's device code is loaded, and right
// again after a device reset between calls). All calls on a device share the
// array: the merge counters that must start at zero are cleared on every
// call, everything else is rewritten by the build; two calls whose work
// overlaps on the GPU race on it.
#include <cstdio>

#include "graph.cuh"

namespace {

using namespace bb;

constexpr size_t SCRATCH_BYTES = BB_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// device address of g_scratch on the current device
bb_status scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return report_error(BB_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    *out = p;
    return BB_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bb_status err(bb_status st, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    return report_error(st, buf);
}

bb_status map_error(uint32_t e) {
    if (e & E_ROWPTR) return report_error(BB_ERR_INVALID_ARG, "rowptr is not a valid CSR row pointer");
    if (e & E_COL) return report_error(BB_ERR_INVALID_ARG, "a column id is outside [0, nV)");
    if (e & E_SIGN) return report_error(BB_ERR_INVALID_ARG, "a sign is not +1 or -1");
    if (e & E_DUP) return report_error(BB_ERR_INVALID_ARG, "an edge is listed twice");
    return err(BB_ERR_CUDA, "internal device check failed (0x%llx)", e);
}

struct Result {
    unsigned long long acc[4];
    uint32_t count_err, build_err;
    unsigned long long wedges;
};

}  // namespace

extern "C" bb_status bb_count_csr_device_noalloc(const bb_csr *csr_dev, const int8_t *signs_dev,
                                                 void *stream, int64_t *balanced, int64_t *total,
                                                 int64_t *wedges_opt) {
    if (!csr_dev || !balanced || !total) return report_error(BB_ERR_INVALID_ARG, "NULL argument");
    const int64_t nU = csr_dev->nU, nV = csr_dev->nV, nE = csr_dev->nE;
    if (nU < 0 || nV < 0 || nE < 0) return report_error(BB_ERR_INVALID_ARG, "negative size");
    if (nU == 0 && nE != 0) return report_error(BB_ERR_INVALID_ARG, "nE must be 0 when nU is 0");
    if (!csr_dev->rowptr || (nE > 0 && (!csr_dev->col || !signs_dev)))
        return report_error(BB_ERR_INVALID_ARG, "rowptr, col or signs is NULL");
    if (nU + nV >= ((int64_t)1 << 31) || nE >= ((int64_t)1 << 32) - 1)
        return report_error(BB_ERR_TOO_LARGE, "graph beyond the id limits");
    const BuildSizes bs = build_sizes(nU, nV, nE, false);  // always the wedge classes
    const size_t need = align256(bs.graph_bytes) + bs.temp_bytes;
    if (need > SCRATCH_BYTES)
        return err(BB_ERR_TOO_LARGE,
                   "graph needs %lld bytes of workspace; the allocation-free entry point has %lld",
                   (long long)need, (long long)SCRATCH_BYTES);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return report_error(BB_ERR_NO_DEVICE, "no current device");
    }
    void *base = nullptr;
    bb_status st = scratch_address(&base);
    if (st != BB_OK) return st;
    count_init();
    cudaStream_t s = (cudaStream_t)stream;
    DevGraph g;
    layout_graph(g, nU, nV, nE, base, false);
    void *temp = (char *)base + align256(bs.graph_bytes);
    // the split-merge counters must start at zero; the array keeps the last call's bytes
    cudaMemsetAsync(g.gpart, 0, (size_t)g.gpart_cap * 4, s);
    cudaMemsetAsync(g.gdone, 0, (size_t)MAX_SPLIT_JOBS * 4, s);
    uint32_t verr = 0;
    st = build_graph(g, csr_dev->rowptr, csr_dev->col, signs_dev, temp, s, nullptr, &verr);
    if (st != BB_OK) return st;
    if ((e = cudaGetLastError()) != cudaSuccess) return report_error(BB_ERR_CUDA, cudaGetErrorString(e));
    if (verr) return map_error(verr);
    launch_count(g, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return report_error(BB_ERR_CUDA, cudaGetErrorString(e));
    // the bounded wait comes first (the library's wait limit); the small
    // copies to pageable host memory then complete at once on the idle stream
    if ((st = wait_stream_bounded(s, "allocation-free count")) != BB_OK) return st;
    Result h;
    e = cudaMemcpyAsync(h.acc, g.scratch->acc, sizeof(h.acc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h.count_err, &g.scratch->err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h.build_err, g.err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h.wedges, g.wedges, 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) { cudaGetLastError(); return report_error(BB_ERR_CUDA, cudaGetErrorString(e)); }
    if (h.build_err) return map_error(h.build_err);
    if (h.count_err) return err(BB_ERR_CUDA, "internal count check failed (0x%llx)", h.count_err);
    if (h.acc[1] || h.acc[3] || h.acc[0] > 0x7fffffffffffffffull || h.acc[2] > 0x7fffffffffffffffull)
        return report_error(BB_ERR_OVERFLOW, "butterfly count exceeds int64");
    *balanced = (int64_t)h.acc[0];
    *total = (int64_t)h.acc[2];
    if (wedges_opt) *wedges_opt = (int64_t)h.wedges;
    return BB_OK;
}
