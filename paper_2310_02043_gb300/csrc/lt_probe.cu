// lt_probe.cu -- L2 read-bandwidth microbenchmark (lt_probe_l2_read in
// include/lt.h): the rate against which the traversal's algorithmic bytes
// are reported. A buffer that fits in L2 is read over and over with 16-byte
// loads that are cached in L2 only (ld.global.cg), so after the first sweep
// every load is an L2 hit; CUDA events time the sweeps.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/lt.h"

namespace {

constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads) l2_read_kernel(const uint4 *__restrict__ buf, uint64_t n_vec,
                                                                int32_t reps, uint32_t *sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int32_t r = 0; r < reps; ++r) {
        uint64_t i = first;
        for (; i + 3 * stride < n_vec; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n_vec; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    // the buffer holds zeros, so this store never happens; it keeps the loads
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

}  // namespace

extern "C" {

int lt_probe_l2_read(int device, uint64_t bytes, int32_t reps, double *gbs_out) {
    if (!gbs_out || reps < 1 || bytes < (1u << 20) || bytes > (uint64_t)96 << 20) return LT_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return LT_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return LT_ERR_ARG;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const uint64_t n_vec = bytes / sizeof(uint4);
    uint4 *buf = nullptr;
    uint32_t *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, n_vec * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, n_vec * sizeof(uint4), s);
    const int grid = sms * 4;
    float best_ms = 0.0f;
    // one warm-up sweep brings the buffer into L2, then the best of 5 timed runs
    if (e == cudaSuccess) {
        l2_read_kernel<<<grid, kProbeThreads, 0, s>>>(buf, n_vec, 1, sink);
        e = cudaGetLastError();
    }
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) l2_read_kernel<<<grid, kProbeThreads, 0, s>>>(buf, n_vec, reps, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best_ms == 0.0f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(buf);
    cudaFree(sink);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA;
    *gbs_out = (double)n_vec * sizeof(uint4) * (double)reps / (best_ms * 1e-3) / 1e9;
    return LT_OK;
}

}  // extern "C"
