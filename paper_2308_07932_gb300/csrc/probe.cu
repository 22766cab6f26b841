// probe.cu - shared-memory atomic throughput on this GPU: the second
// ceiling of the wedge kernels, whose inner step is one shared-memory
// atomicAdd on a packed (symmetric, asymmetric) counter whose previous
// value is used. Each thread adds to pseudo-random counters of a window
// (an LCG picks the index) and folds the returned values into a sum, so
// the atomics cannot be dropped or turned into reductions.
#include <algorithm>

#include "runtime.h"

namespace {

constexpr int PROBE_THREADS = 512;
constexpr int PROBE_ITERS = 2048;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_atomics(uint32_t window, uint32_t seed,
                                                                 unsigned long long *sink) {
    extern __shared__ uint32_t cnt[];
    for (uint32_t i = threadIdx.x; i < window; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    uint32_t x = seed ^ (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u;
    uint32_t acc = 0;
#pragma unroll 4
    for (int k = 0; k < PROBE_ITERS; k++) {
        x = x * 1664525u + 1013904223u;
        const uint32_t idx = (uint32_t)(((uint64_t)x * window) >> 32);
        acc += atomicAdd(&cnt[idx], (x & 0x100u) ? (1u << 16) : 1u);
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps acc live; practically never taken
}

}  // namespace

extern "C" bb_status bb_probe_shared_atomics(int device, uint32_t window, double *atomics_per_s) {
    using namespace bb;
    if (!atomics_per_s || window < 32 || window > 49152)
        return fail(BB_ERR_INVALID_ARG, "window %u outside [32, 49152] or NULL output", window);
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return fail(BB_ERR_NO_DEVICE, "no CUDA device %d", device);
    }
    BB_CUDA(cudaSetDevice(device), "cudaSetDevice");
    cudaDeviceProp prop;
    BB_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    const size_t smem = (size_t)window * 4;
    BB_CUDA(cudaFuncSetAttribute(k_probe_atomics, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "probe attribute");
    int per_sm = 0;
    BB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_atomics, PROBE_THREADS, smem),
            "probe occupancy");
    const int blocks = std::max(1, per_sm) * prop.multiProcessorCount * 4;
    cudaStream_t s;
    BB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    unsigned long long *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sink, 8, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {  // first run warms up
        cudaEventRecord(e0, s);
        k_probe_atomics<<<blocks, PROBE_THREADS, smem, s>>>(window, 12345u + rep, sink);
        note_launch();
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            bb_status st = wait_bounded(s, "atomic probe");
            if (st != BB_OK) { cudaStreamDestroy(s); return st; }
        }
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0 || ms < best)) best = ms;
    }
    if (sink) cudaFreeAsync(sink, s);
    const bb_status ws = wait_bounded(s, "atomic probe");
    if (ws != BB_OK) return ws;  // the stream and events stay (leaked) while work runs
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(e, "atomic probe");
    *atomics_per_s = (double)blocks * PROBE_THREADS * PROBE_ITERS / (best / 1e3);
    return BB_OK;
}
