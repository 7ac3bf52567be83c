// lt_noalloc.cu -- the objective and adjoint weights for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc at all: code running inside a
// memory pool that another framework owns (its allocator would not see the
// block and could not account for it), or on a device already filled to its
// budget. lt_loss_static computes the same objective as lt_loss from buffers
// the caller owns, and keeps its only scratch -- one partial sum per block --
// in a fixed array compiled into this library.
#include <cstdint>
#include <mutex>

#include "../../include/lt.h"

namespace {

constexpr int kThreads = 256;
constexpr int kTexelsPerThread = 16;
constexpr int64_t kTexelsPerBlock = (int64_t)kThreads * kTexelsPerThread;   // 4096
constexpr int kMaxBlocks = 4096;                                             // 32 KiB of partials
static_assert((int64_t)kMaxBlocks * kTexelsPerBlock == LT_LOSS_STATIC_MAX_TEXELS, "limit in lt.h");
constexpr int kMaxDevices = 64;

// Block partial sums of the objective. Every device that loads the library
// holds this array until the process exits; all calls on a device share it.
static __device__ __align__(256) double g_loss_partials[kMaxBlocks];

// Host-side address of g_loss_partials on each device, looked up once.
std::mutex g_mutex;
double *g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) t += sh[i];
    __syncthreads();
    return t;
}

// Block b handles texels [b * 4096, (b + 1) * 4096); its partial sum of
// 1/2 A_t alpha_t (E_t - E*_t)^2 goes to partial[b].
__global__ void __launch_bounds__(kThreads) loss_blocks_kernel(const long long *q, double inv_scale,
                                                               const float *area, const float *E_target,
                                                               const float *alpha, int64_t n, float *w_out,
                                                               float *E_out, double *partial) {
    __shared__ double sh[kThreads / 32];
    double part = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kTexelsPerBlock;
    for (int i = 0; i < kTexelsPerThread; ++i) {
        const int64_t t = base + (int64_t)i * kThreads + threadIdx.x;
        if (t >= n) break;
        const double A = (double)area[t];
        const double E = (double)q[t] * inv_scale / A;
        const double r = E - (double)E_target[t];
        const double a = alpha ? (double)alpha[t] : 1.0;
        if (E_out) E_out[t] = (float)E;
        w_out[t] = (float)(a * r);
        part += 0.5 * A * a * r * r;
    }
    const double s = block_sum(part, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) loss_sum_kernel(const double *partial, int n, double *out) {
    __shared__ double sh[kThreads / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) v += partial[i];
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) *out = s;
}

// Device address of the partials array on `device` (which must be current).
// Locking a mutex may throw std::system_error; that stays on this side of
// the C ABI as a CUDA-style error.
cudaError_t partials_on(int device, double **out) noexcept {
    try {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_partials_addr[device]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_loss_partials);
            if (e != cudaSuccess) return e;
            g_partials_addr[device] = static_cast<double *>(p);
        }
        *out = g_partials_addr[device];
        return cudaSuccess;
    } catch (...) {
        return cudaErrorUnknown;
    }
}

}  // namespace

extern "C" int lt_loss_static(int device, void *cuda_stream, const int64_t *q, double scale, const float *area,
                              const float *E_target, const float *alpha, int64_t n_texels, float *w_out,
                              float *E_out, double *loss_out) {
    if (device < 0 || device >= kMaxDevices || !q || !area || !E_target || !w_out || !loss_out || !(scale > 0.0))
        return LT_ERR_ARG;
    if (n_texels < 1 || n_texels > LT_LOSS_STATIC_MAX_TEXELS) return LT_ERR_ARG;
    // An error left pending by earlier, unrelated CUDA work would be reported
    // as this call's launch failure; refuse instead, and leave it pending.
    if (cudaPeekAtLastError() != cudaSuccess) return LT_ERR_STATE;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return LT_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return LT_ERR_CUDA;
    double *partial = nullptr;
    cudaError_t e = partials_on(device, &partial);
    if (e == cudaSuccess) {
        const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        const int blocks = (int)((n_texels + kTexelsPerBlock - 1) / kTexelsPerBlock);
        loss_blocks_kernel<<<blocks, kThreads, 0, s>>>(reinterpret_cast<const long long *>(q), 1.0 / scale, area,
                                                       E_target, alpha, n_texels, w_out, E_out, partial);
        loss_sum_kernel<<<1, kThreads, 0, s>>>(partial, blocks, loss_out);
        e = cudaGetLastError();
    }
    if (prev != device) cudaSetDevice(prev);
    return e == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}
