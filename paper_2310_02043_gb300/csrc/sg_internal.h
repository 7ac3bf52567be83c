// sg_internal.h -- device layouts and launchers of the irradiance surrogate
// (sg_kernels.cu), used by its C ABI (sg_api.cpp).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace sg {

constexpr int kLevels = 16;
constexpr int kTableLog2 = 19;
constexpr int kTableSize = 1 << kTableLog2;
constexpr int kIn = 64, kHid = 64, kOut = 16;
constexpr int kOffW0 = 0, kOffW1 = 64 * 64, kOffW2 = 2 * 64 * 64, kOffW3 = 3 * 64 * 64;
constexpr int kWeights = 3 * 64 * 64 + 16 * 64;
constexpr int64_t kTableFloats = (int64_t)kLevels * kTableSize * 2;
constexpr int kGeom = 17;           // input entries 32..48
constexpr int kMlpWarps = 8;        // warps per block of the network kernels
constexpr int kWgradChunk = 4096;   // rows per block of the weight-gradient kernel
constexpr int kWgradItems = 13;     // (layer 0..2) x 4 row tiles of dW, + layer 3

// Per-light constants, derived on the host in double.
struct alignas(16) LightC {
    float p[3];
    float intensity;          // I = p_int^2 / 2
    float nl[3];
    float p_int;
    float dny[3];             // dn/dyaw
    float ci;                 // cos(theta_in)
    float dnp[3];             // dn/dpitch
    float co;                 // cos(theta_out)
    float inv_dc;             // 1 / (ci - co)
    float sin_in;
    float pad[2];
};
static_assert(sizeof(LightC) == 80, "light layout");

struct TexelView {
    const float4 *pos;        // [T_pad] centre (w unused)
    const float4 *nrm;        // [T_pad] unit normal
    const float *area;        // [T_pad], 0 on padding
    int64_t n;                // texels
    int64_t n_pad;            // multiple of 16
    float lo[3];
    float inv_ext;            // float32 1 / ext
    float ext;
    float inv_mean_area;
};

// Buffers of a batch of network rows kept for the weight gradient.
struct RowBuffers {
    uint16_t *act;            // [4][rows][64] bf16 inputs of the four products
    uint16_t *dz;             // [3][rows][64] bf16 gradients at z1..z3, then [rows][16] at o
    int32_t rows;             // capacity (multiple of 16)
};

struct TrainArgs {
    TexelView tex;
    const LightC *lights;     // [solves]
    int32_t n_solves;
    const float *E_obs;       // [solves][n]
    const int32_t *samples;   // [batch][2] or null (drawn from seed, step)
    uint64_t seed, step;
    int32_t batch;
    const float *table;       // fp32 [16][2^19][2]
    float *dtable;            // gradient, zeroed before the launch
    const uint16_t *Wb;       // bf16 weights
    RowBuffers rb;
    double *loss_part;        // [grid]
};

struct NetworkArgs {
    const float *X;           // [rows][64]
    const float *dO;          // [rows][16] or null
    int32_t rows;
    const uint16_t *Wb;
    float *O;                 // [rows][16]
    float *dX;                // [rows][64] or null
    RowBuffers rb;
};

struct DesignArgs {
    TexelView tex;
    const LightC *lights;
    int32_t n_lights;
    const uint16_t *enc;      // [T_pad][32] bf16 encoding of every texel
    const uint16_t *Wb;
    float *K;                 // [lights][T_pad]
    const float *up;          // [T_pad] A_t w_t (backward)
    float *gpart;             // [lights][T_pad / 16][8] (backward)
};

// The fused design objective (one kernel for forward, per-texel irradiance,
// objective, weights and backward) serves designs of at most this many lights.
constexpr int kFusedMaxLights = 32;
struct FusedArgs {
    const float *target;      // [n] E*
    const float *alpha;       // [n] or null (ones)
    float *E_out;             // [n] or null
    double *loss_part;        // [grid] objective partials
    int32_t texels_per_tile;  // 128 / n_lights
    int64_t n_tiles;          // ceil(n_pad / texels_per_tile); gpart is [lights][n_tiles][8]
};
cudaError_t launch_design_fused_tc(const DesignArgs &a, const FusedArgs &f, int32_t *err, cudaStream_t s,
                                   int *grid_out);

cudaError_t launch_train(const TrainArgs &a, int grid, cudaStream_t s);
// tcgen05 training kernel; *grid_out = its grid (the number of loss partials)
cudaError_t launch_train_tc(const TrainArgs &a, int32_t *err, cudaStream_t s, int *grid_out);
cudaError_t launch_network(const NetworkArgs &a, cudaStream_t s);
// Weight gradient of `rows` kept rows: partial sums per chunk, then their
// ordered sum into dW [kWeights]; loss partials (if any) summed into *loss.
cudaError_t launch_wgrad(const RowBuffers &rb, int32_t rows, float *partial, float *dW, const double *loss_part,
                         int32_t n_loss_part, double *loss, cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, uint16_t *bf16_out, cudaStream_t s);
cudaError_t launch_encode_points(const float *xn, int32_t n, const float *table, float *enc_out, cudaStream_t s);
cudaError_t launch_encode_texels(const TexelView &t, const float *table, uint16_t *enc, cudaStream_t s);
cudaError_t launch_design_forward(const DesignArgs &a, cudaStream_t s);
// The same on tcgen05 (TMEM accumulators); err gets bit 1 if a wait gave up.
cudaError_t launch_design_forward_tc(const DesignArgs &a, int32_t *err, cudaStream_t s);
cudaError_t launch_design_reduce(const TexelView &t, const LightC *lights, int32_t n_lights, const float *K,
                                 const float *E_target, const float *alpha, float *E_out, float *up,
                                 double *loss_part, cudaStream_t s);
cudaError_t launch_design_backward(const DesignArgs &a, cudaStream_t s);
cudaError_t launch_design_backward_tc(const DesignArgs &a, int32_t *err, cudaStream_t s);
// Per-light sums of gpart [lights][tiles_per_light][8] and the objective (the
// sum of n_loss_part partials; 0 = those of launch_design_reduce).
cudaError_t launch_design_final(const float *gpart, const LightC *lights, int32_t n_lights, int64_t tiles_per_light,
                                const double *loss_part, int32_t n_loss_part, double *out, cudaStream_t s);
int train_grid(int device);
constexpr int kReduceBlocks = 256;   // blocks of the design reduce kernel (loss partials)

}  // namespace sg
