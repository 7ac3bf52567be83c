// sg_kernels.cu -- kernels of the irradiance surrogate: hash encoding, a fused
// 4 x 64 network on the tensor cores (mma.sync m16n8k16, bf16 inputs, fp32
// accumulation; each warp carries 16 rows through all layers in registers),
// its weight gradient, Adam, and the design objective with its gradient with
// respect to the luminaire parameters.
#include <algorithm>

#include <cuda_bf16.h>

#include "sg_internal.h"

namespace sg {
namespace {

__constant__ int c_res[kLevels] = {16, 20, 25, 32, 40, 50, 64, 80, 101, 128, 161, 203, 256, 322, 406, 512};
constexpr int kDenseLevels = 7;            // levels whose (N+1)^3 grid fits 2^19 entries
constexpr float kRScale = 0.01f;
constexpr int LDW = 72;                    // row stride (elements) of 64-wide bf16 rows in shared memory
constexpr int LDT3 = 24;                   // row stride of W3 transposed ([64][16])
constexpr int S_W0 = 0, S_W1 = S_W0 + 64 * LDW, S_W2 = S_W1 + 64 * LDW, S_W3 = S_W2 + 64 * LDW;
constexpr int S_T0 = S_W3 + 16 * LDW, S_T1 = S_T0 + 64 * LDW, S_T2 = S_T1 + 64 * LDW, S_T3 = S_T2 + 64 * LDW;
constexpr int S_FWD_END = S_T0;            // forward-only kernels stop here
constexpr int S_ALL_END = S_T3 + 64 * LDT3;

// Per-warp scratch after the weights.
struct alignas(16) WarpScratch {
    uint16_t X[16 * LDW];     // bf16 input rows
    float D[16];
    float aux0[16];           // E_obs (train) or gD (design backward)
    float aux1[16];           // loss weight (train) or A w K (design backward)
    float xn[16][3];
    int32_t sidx[16], tidx[16];
    float gX[16][kGeom];
};

constexpr size_t smem_bytes(bool transposed) {
    return (size_t)(transposed ? S_ALL_END : S_FWD_END) * 2 + (size_t)kMlpWarps * sizeof(WarpScratch);
}

// ---------------------------------------------------------------------------
// tensor-core helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld32(const uint16_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    __nv_bfloat16 v = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t *>(&v);
}

__device__ __forceinline__ float lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_f(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// Weights into shared memory: W_k as [out][LDW] (forward operand) and, if
// requested, transposed as [in][LDW] / [64][LDT3] (backward operand).
__device__ void load_weights(uint16_t *s, const uint16_t *__restrict__ W, bool transposed) {
    for (int i = threadIdx.x; i < kWeights; i += blockDim.x) {
        const uint16_t v = W[i];
        if (i < kOffW3) {
            const int layer = i >> 12, r = i & 4095, n = r >> 6, m = r & 63;
            s[S_W0 + layer * 64 * LDW + n * LDW + m] = v;
            if (transposed) s[S_T0 + layer * 64 * LDW + m * LDW + n] = v;
        } else {
            const int r = i - kOffW3, n = r >> 6, m = r & 63;
            s[S_W3 + n * LDW + m] = v;
            if (transposed) s[S_T3 + m * LDT3 + n] = v;
        }
    }
}

// A fragments (16 x 64, four k-tiles) of the bf16 rows in X.
__device__ __forceinline__ void load_rows(uint32_t (&A)[4][4], const uint16_t *X, int g, int c) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        A[kk][0] = ld32(X + g * LDW + 16 * kk + 2 * c);
        A[kk][1] = ld32(X + (g + 8) * LDW + 16 * kk + 2 * c);
        A[kk][2] = ld32(X + g * LDW + 16 * kk + 8 + 2 * c);
        A[kk][3] = ld32(X + (g + 8) * LDW + 16 * kk + 8 + 2 * c);
    }
}

// acc (16 x 64) = A (16 x 64) B, B[k][n] = M[n][k] with M in shared memory
// as [64][LDW] rows.
__device__ __forceinline__ void gemm64(float (&acc)[8][4], const uint32_t (&A)[4][4], const uint16_t *M, int g, int c) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint16_t *w = M + (8 * j + g) * LDW + 16 * kk + 2 * c;
            mma(acc[j], A[kk], ld32(w), ld32(w + 8));
        }
    }
}

// Accumulator tiles -> bf16 A fragments of relu(acc).
__device__ __forceinline__ void relu_pack(const float (&acc)[8][4], uint32_t (&A)[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float *t = acc[2 * kk + h];
            A[kk][2 * h] = pack2(fmaxf(t[0], 0.0f), fmaxf(t[1], 0.0f));
            A[kk][2 * h + 1] = pack2(fmaxf(t[2], 0.0f), fmaxf(t[3], 0.0f));
        }
}

// Gradient tiles times the ReLU mask of the forward activations -> bf16 A
// fragments (the gradient at the pre-activation, rounded for the next product).
__device__ __forceinline__ void mask_pack(const float (&acc)[8][4], const uint32_t (&act)[4][4], uint32_t (&G)[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float *t = acc[2 * kk + h];
            const uint32_t a0 = act[kk][2 * h], a1 = act[kk][2 * h + 1];
            G[kk][2 * h] = pack2(lo_f(a0) > 0.0f ? t[0] : 0.0f, hi_f(a0) > 0.0f ? t[1] : 0.0f);
            G[kk][2 * h + 1] = pack2(lo_f(a1) > 0.0f ? t[2] : 0.0f, hi_f(a1) > 0.0f ? t[3] : 0.0f);
        }
}

// Fragments -> rows [rows][64] bf16 in global memory.
__device__ __forceinline__ void store_frags(uint16_t *base, int64_t row0, const uint32_t (&A)[4][4], int g, int c) {
    uint32_t *b = reinterpret_cast<uint32_t *>(base);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        b[(row0 + g) * 32 + 8 * kk + c] = A[kk][0];
        b[(row0 + g + 8) * 32 + 8 * kk + c] = A[kk][1];
        b[(row0 + g) * 32 + 8 * kk + 4 + c] = A[kk][2];
        b[(row0 + g + 8) * 32 + 8 * kk + 4 + c] = A[kk][3];
    }
}

__device__ __forceinline__ void store_dO(uint16_t *base, int64_t row0, const uint32_t (&a)[4], int g, int c) {
    uint32_t *b = reinterpret_cast<uint32_t *>(base);
    b[(row0 + g) * 8 + c] = a[0];
    b[(row0 + g + 8) * 8 + c] = a[1];
    b[(row0 + g) * 8 + 4 + c] = a[2];
    b[(row0 + g + 8) * 8 + 4 + c] = a[3];
}

// Forward of 16 rows: act[k] = bf16 inputs of products 1..3, o = output tiles.
__device__ __forceinline__ void forward(const uint16_t *sw, const uint16_t *X, uint32_t (&act)[3][4][4],
                                        float (&o)[2][4], int g, int c) {
    uint32_t A0[4][4];
    load_rows(A0, X, g, c);
    float acc[8][4];
    gemm64(acc, A0, sw + S_W0, g, c);
    relu_pack(acc, act[0]);
    gemm64(acc, act[0], sw + S_W1, g, c);
    relu_pack(acc, act[1]);
    gemm64(acc, act[1], sw + S_W2, g, c);
    relu_pack(acc, act[2]);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        o[j][0] = o[j][1] = o[j][2] = o[j][3] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint16_t *w = sw + S_W3 + (8 * j + g) * LDW + 16 * kk + 2 * c;
            mma(o[j], act[2][kk], ld32(w), ld32(w + 8));
        }
    }
}

// Backward of 16 rows from the output gradient fragment dO (one k-tile of
// the 16 outputs): dX = gradient at the input (fp32 tiles). If dz is set,
// the bf16 gradients at z3, z2, z1 are stored as rows of dz[0..2].
__device__ __forceinline__ void backward(const uint16_t *sw, const uint32_t (&act)[3][4][4], const uint32_t (&dO)[4],
                                         float (&dX)[8][4], int g, int c, uint16_t *dz, int64_t rows_cap,
                                         int64_t row0) {
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
        const uint16_t *w = sw + S_T3 + (8 * j + g) * LDT3 + 2 * c;
        mma(acc[j], dO, ld32(w), ld32(w + 8));
    }
    uint32_t G[4][4];
    mask_pack(acc, act[2], G);
    if (dz) store_frags(dz + 2 * rows_cap * 64, row0, G, g, c);
    gemm64(acc, G, sw + S_T2, g, c);
    mask_pack(acc, act[1], G);
    if (dz) store_frags(dz + 1 * rows_cap * 64, row0, G, g, c);
    gemm64(acc, G, sw + S_T1, g, c);
    mask_pack(acc, act[0], G);
    if (dz) store_frags(dz, row0, G, g, c);
    gemm64(dX, G, sw + S_T0, g, c);
}

// ---------------------------------------------------------------------------
// hash encoding
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cell_of(const float (&xn)[3], int level, int (&i0)[3], float (&f)[3]) {
    const float n = (float)c_res[level];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float pos = __fmul_rn(xn[a], n);
        int ii = (int)floorf(pos);
        ii = min(max(ii, 0), c_res[level] - 1);
        f[a] = fminf(fmaxf(__fsub_rn(pos, (float)ii), 0.0f), 1.0f);
        i0[a] = ii;
    }
}

__device__ __forceinline__ uint32_t vertex_index(int level, int x, int y, int z) {
    if (level < kDenseLevels) {
        const uint32_t n = (uint32_t)c_res[level] + 1u;
        return (uint32_t)x + n * ((uint32_t)y + n * (uint32_t)z);
    }
    return ((uint32_t)x ^ ((uint32_t)y * 2654435761u) ^ ((uint32_t)z * 805459861u)) & (uint32_t)(kTableSize - 1);
}

__device__ __forceinline__ float2 encode_level(const float (&xn)[3], int level, const float *__restrict__ table) {
    int i0[3];
    float f[3];
    cell_of(xn, level, i0, f);
    const float2 *tl = reinterpret_cast<const float2 *>(table) + (size_t)level * kTableSize;
    float2 e = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int cn = 0; cn < 8; ++cn) {
        const int bx = cn & 1, by = (cn >> 1) & 1, bz = (cn >> 2) & 1;
        const float w = (bx ? f[0] : 1.0f - f[0]) * (by ? f[1] : 1.0f - f[1]) * (bz ? f[2] : 1.0f - f[2]);
        const float2 v = __ldg(tl + vertex_index(level, i0[0] + bx, i0[1] + by, i0[2] + bz));
        e.x += w * v.x;
        e.y += w * v.y;
    }
    return e;
}

__device__ __forceinline__ void scatter_level(const float (&xn)[3], int level, float g0, float g1, float *dtable) {
    if (g0 == 0.0f && g1 == 0.0f) return;
    int i0[3];
    float f[3];
    cell_of(xn, level, i0, f);
    float *tl = dtable + (size_t)level * kTableSize * 2;
#pragma unroll
    for (int cn = 0; cn < 8; ++cn) {
        const int bx = cn & 1, by = (cn >> 1) & 1, bz = (cn >> 2) & 1;
        const float w = (bx ? f[0] : 1.0f - f[0]) * (by ? f[1] : 1.0f - f[1]) * (bz ? f[2] : 1.0f - f[2]);
        const uint32_t idx = vertex_index(level, i0[0] + bx, i0[1] + by, i0[2] + bz);
        // both features of the entry in one vector atomic (8-byte aligned)
        atomicAdd(reinterpret_cast<float2 *>(tl) + idx, make_float2(w * g0, w * g1));
    }
}

__device__ __forceinline__ void normalised(const TexelView &tv, float4 P, float (&xn)[3]) {
    xn[0] = __fmul_rn(__fsub_rn(P.x, tv.lo[0]), tv.inv_ext);
    xn[1] = __fmul_rn(__fsub_rn(P.y, tv.lo[1]), tv.inv_ext);
    xn[2] = __fmul_rn(__fsub_rn(P.z, tv.lo[2]), tv.inv_ext);
}

// ---------------------------------------------------------------------------
// geometric light features (input entries 32..48) and their gradient
// ---------------------------------------------------------------------------
struct Geo {
    float ux, uy, uz, r, r2, ir, cl, cr, acr, a, s;
    bool soft;
};

__device__ __forceinline__ Geo geo_of(const LightC &L, float4 P, float4 N) {
    Geo q;
    const float dx = L.p[0] - P.x, dy = L.p[1] - P.y, dz = L.p[2] - P.z;
    q.r2 = dx * dx + dy * dy + dz * dz;
    q.r = sqrtf(q.r2);
    q.ir = 1.0f / q.r;
    q.ux = dx * q.ir;
    q.uy = dy * q.ir;
    q.uz = dz * q.ir;
    q.cl = -(q.ux * L.nl[0] + q.uy * L.nl[1] + q.uz * L.nl[2]);
    q.cr = N.x * q.ux + N.y * q.uy + N.z * q.uz;
    q.acr = fabsf(q.cr);
    q.s = (q.cl - L.co) * L.inv_dc;
    q.soft = q.cl > L.co && q.cl < L.ci;
    q.a = q.cl >= L.ci ? 1.0f : (q.soft ? q.s * q.s : 0.0f);
    return q;
}

// Writes entries 32..63 of one input row (bf16) and returns D.
__device__ __forceinline__ float geometry_row(const LightC &L, float4 P, float4 N, const TexelView &tv, uint16_t *row) {
    const Geo q = geo_of(L, P, N);
    float G[kGeom];
    G[0] = q.ux;
    G[1] = q.uy;
    G[2] = q.uz;
    G[3] = q.r * 0.1f;
    G[4] = L.nl[0];
    G[5] = L.nl[1];
    G[6] = L.nl[2];
    G[7] = q.cl;
    G[8] = q.acr;
    G[9] = q.a;
    G[10] = L.ci;
    G[11] = (L.p[0] - tv.lo[0]) * tv.inv_ext;
    G[12] = (L.p[1] - tv.lo[1]) * tv.inv_ext;
    G[13] = (L.p[2] - tv.lo[2]) * tv.inv_ext;
    G[14] = N.x;
    G[15] = N.y;
    G[16] = N.z;
#pragma unroll
    for (int k = 0; k < kGeom; ++k) row[32 + k] = bf16_bits(G[k]);
    row[49] = bf16_bits(1.0f);
#pragma unroll
    for (int k = 50; k < 64; ++k) row[k] = 0;
    return q.a * q.acr / q.r2;
}

// dO/d(x, y, z, yaw, pitch, theta_in) of one row from the gradient at the
// input entries 32..48 (gX) and at D (gD), by the chain rule through the
// features.
__device__ __forceinline__ void geometry_grad(const LightC &L, float4 P, float4 N, const TexelView &tv,
                                              const float *gX, float gD, float (&g)[6]) {
    const Geo q = geo_of(L, P, N);
    const float da_dcos = q.soft ? 2.0f * q.s * L.inv_dc : 0.0f;
    const float da_dthin = q.soft ? 2.0f * q.s * q.s * L.inv_dc * L.sin_in : 0.0f;
    const float g_a = gX[9] + gD * q.acr / q.r2;
    const float g_cl = gX[7] + g_a * da_dcos;
    const float g_cr = gX[8] + gD * q.a / q.r2;
    const float sg = q.cr > 0.0f ? 1.0f : (q.cr < 0.0f ? -1.0f : 0.0f);
    const float vx = gX[0] - L.nl[0] * g_cl + sg * N.x * g_cr;
    const float vy = gX[1] - L.nl[1] * g_cl + sg * N.y * g_cr;
    const float vz = gX[2] - L.nl[2] * g_cl + sg * N.z * g_cr;
    const float udv = q.ux * vx + q.uy * vy + q.uz * vz;
    const float radial = gX[3] * 0.1f - 2.0f * gD * q.a * q.acr / (q.r2 * q.r);
    g[0] = (vx - q.ux * udv) * q.ir + q.ux * radial + gX[11] * tv.inv_ext;
    g[1] = (vy - q.uy * udv) * q.ir + q.uy * radial + gX[12] * tv.inv_ext;
    g[2] = (vz - q.uz * udv) * q.ir + q.uz * radial + gX[13] * tv.inv_ext;
    const float u_dny = q.ux * L.dny[0] + q.uy * L.dny[1] + q.uz * L.dny[2];
    const float u_dnp = q.ux * L.dnp[0] + q.uy * L.dnp[1] + q.uz * L.dnp[2];
    g[3] = gX[4] * L.dny[0] + gX[5] * L.dny[1] + gX[6] * L.dny[2] - g_cl * u_dny;
    g[4] = gX[4] * L.dnp[0] + gX[5] * L.dnp[1] + gX[6] * L.dnp[2] - g_cl * u_dnp;
    g[5] = g_a * da_dthin - gX[10] * L.sin_in;
}

__device__ __forceinline__ float sigmoidf_(float v) { return 1.0f / (1.0f + __expf(-v)); }
__device__ __forceinline__ float softplusf_(float v) { return v > 20.0f ? v : log1pf(__expf(v)); }

// splitmix64 (Steele, Lea and Flood 2014) for drawing training samples.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMlpWarps * 32, 2) train_kernel(const TrainArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *sw = reinterpret_cast<uint16_t *>(smem_raw);
    __shared__ double red[kMlpWarps];
    load_weights(sw, A.Wb, true);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    WarpScratch *ws = reinterpret_cast<WarpScratch *>(smem_raw + (size_t)S_ALL_END * 2) + warp;
    const int64_t n = A.tex.n;
    const int64_t tiles = ((int64_t)A.batch + 15) / 16;
    const int64_t cap = A.rb.rows;
    const double inv_b = 1.0 / (double)A.batch;
    double loss = 0.0;
    for (int64_t tile = (int64_t)blockIdx.x * kMlpWarps + warp; tile < tiles; tile += (int64_t)gridDim.x * kMlpWarps) {
        const int64_t row0 = tile * 16;
        if (lane < 16) {
            const int64_t i = row0 + lane;
            const bool valid = i < A.batch;
            int32_t s = 0, t = 0;
            if (valid) {
                if (A.samples) {
                    s = A.samples[2 * i];
                    t = A.samples[2 * i + 1];
                } else {
                    const uint64_t r = mix64(A.seed ^ mix64((A.step << 32) ^ (uint64_t)i));
                    s = (int32_t)(((r >> 32) * (uint64_t)A.n_solves) >> 32);
                    t = (int32_t)(((r & 0xFFFFFFFFull) * (uint64_t)n) >> 32);
                }
            }
            const float4 P = A.tex.pos[t], N = A.tex.nrm[t];
            uint16_t *row = ws->X + lane * LDW;
            ws->D[lane] = geometry_row(A.lights[s], P, N, A.tex, row);
            ws->aux0[lane] = valid ? __ldg(A.E_obs + (int64_t)s * n + t) : 0.0f;
            ws->aux1[lane] = valid ? A.tex.area[t] * A.tex.inv_mean_area : 0.0f;
            float xn[3];
            normalised(A.tex, P, xn);
            ws->xn[lane][0] = xn[0];
            ws->xn[lane][1] = xn[1];
            ws->xn[lane][2] = xn[2];
            ws->sidx[lane] = s;
            ws->tidx[lane] = valid ? t : -1;
        }
        __syncwarp();
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const int r = lane & 15, level = (lane >> 4) + 2 * p;
            const float xn[3] = {ws->xn[r][0], ws->xn[r][1], ws->xn[r][2]};
            const float2 e = encode_level(xn, level, A.table);
            *reinterpret_cast<uint32_t *>(ws->X + r * LDW + 2 * level) = pack2(e.x, e.y);
        }
        __syncwarp();
        {   // rows of the first product's input
            const uint32_t *src = reinterpret_cast<const uint32_t *>(ws->X);
            uint32_t *dst = reinterpret_cast<uint32_t *>(A.rb.act);
            for (int k = lane; k < 16 * 32; k += 32) dst[(row0 + (k >> 5)) * 32 + (k & 31)] = src[(k >> 5) * (LDW / 2) + (k & 31)];
        }
        uint32_t act[3][4][4];
        float o[2][4];
        forward(sw, ws->X, act, o, g, c);
        store_frags(A.rb.act + 1 * cap * 64, row0, act[0], g, c);
        store_frags(A.rb.act + 2 * cap * 64, row0, act[1], g, c);
        store_frags(A.rb.act + 3 * cap * 64, row0, act[2], g, c);
        uint32_t dO[4] = {0u, 0u, 0u, 0u};
        if (c == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                const float o0 = o[0][2 * h], o1 = o[0][2 * h + 1];
                const float v = sigmoidf_(o0), sp = softplusf_(o1);
                const float D = ws->D[r];
                const float K = v * D + kRScale * sp;
                const float e = K - ws->aux0[r];
                const float wgt = ws->aux1[r];
                loss += 0.5 * (double)wgt * (double)e * (double)e * inv_b;
                const float dK = (float)((double)(wgt * e) * inv_b);
                dO[h] = pack2(dK * v * (1.0f - v) * D, dK * kRScale * sigmoidf_(o1));
            }
        }
        store_dO(A.rb.dz + 3 * cap * 64, row0, dO, g, c);
        float dX[8][4];
        backward(sw, act, dO, dX, g, c, A.rb.dz, cap, row0);
        // encoding gradient: tile j < 4 holds input entries 8j + 2c (+1) = level 4j + c
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                if (ws->tidx[r] < 0) continue;
                const float xn[3] = {ws->xn[r][0], ws->xn[r][1], ws->xn[r][2]};
                scatter_level(xn, 4 * j + c, dX[j][2 * h], dX[j][2 * h + 1], A.dtable);
            }
        __syncwarp();
    }
    loss = warp_sum_d(loss);
    if (lane == 0) red[warp] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kMlpWarps; ++w) s += red[w];
        A.loss_part[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// the network on given rows
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMlpWarps * 32, 2) network_kernel(const NetworkArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *sw = reinterpret_cast<uint16_t *>(smem_raw);
    load_weights(sw, A.Wb, A.dO != nullptr);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    WarpScratch *ws = reinterpret_cast<WarpScratch *>(smem_raw + (size_t)S_ALL_END * 2) + warp;
    const int64_t tiles = ((int64_t)A.rows + 15) / 16;
    const int64_t cap = A.rb.rows;
    for (int64_t tile = (int64_t)blockIdx.x * kMlpWarps + warp; tile < tiles; tile += (int64_t)gridDim.x * kMlpWarps) {
        const int64_t row0 = tile * 16;
        for (int k = lane; k < 16 * 64; k += 32) {
            const int64_t r = row0 + (k >> 6);
            ws->X[(k >> 6) * LDW + (k & 63)] = r < A.rows ? bf16_bits(A.X[r * 64 + (k & 63)]) : (uint16_t)0;
        }
        __syncwarp();
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(ws->X);
            uint32_t *dst = reinterpret_cast<uint32_t *>(A.rb.act);
            for (int k = lane; k < 16 * 32; k += 32) dst[(row0 + (k >> 5)) * 32 + (k & 31)] = src[(k >> 5) * (LDW / 2) + (k & 31)];
        }
        uint32_t act[3][4][4];
        float o[2][4];
        forward(sw, ws->X, act, o, g, c);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t r = row0 + g + 8 * (e >> 1);
                if (r < A.rows) A.O[r * 16 + 8 * j + 2 * c + (e & 1)] = o[j][e];
            }
        if (A.dO) {
            store_frags(A.rb.act + 1 * cap * 64, row0, act[0], g, c);
            store_frags(A.rb.act + 2 * cap * 64, row0, act[1], g, c);
            store_frags(A.rb.act + 3 * cap * 64, row0, act[2], g, c);
            auto dv = [&](int64_t r, int col) { return r < A.rows ? A.dO[r * 16 + col] : 0.0f; };
            uint32_t dO[4];
            dO[0] = pack2(dv(row0 + g, 2 * c), dv(row0 + g, 2 * c + 1));
            dO[1] = pack2(dv(row0 + g + 8, 2 * c), dv(row0 + g + 8, 2 * c + 1));
            dO[2] = pack2(dv(row0 + g, 8 + 2 * c), dv(row0 + g, 9 + 2 * c));
            dO[3] = pack2(dv(row0 + g + 8, 8 + 2 * c), dv(row0 + g + 8, 9 + 2 * c));
            store_dO(A.rb.dz + 3 * cap * 64, row0, dO, g, c);
            float dX[8][4];
            backward(sw, act, dO, dX, g, c, A.rb.dz, cap, row0);
            if (A.dX)
#pragma unroll
                for (int j = 0; j < 8; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int64_t r = row0 + g + 8 * (e >> 1);
                        if (r < A.rows) A.dX[r * 64 + 8 * j + 2 * c + (e & 1)] = dX[j][e];
                    }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW_k = sum over rows of dz_{k+1}^T a_k, per chunk of rows
// ---------------------------------------------------------------------------
struct alignas(16) WgradScratch {
    uint16_t dzs[16 * 24];
    uint16_t as[16 * LDW];
};

__global__ void __launch_bounds__(128) wgrad_kernel(const RowBuffers rb, int32_t rows, float *__restrict__ partial) {
    __shared__ WgradScratch scr[4];
    __shared__ float red[4][16 * 64];
    const int item = blockIdx.y, chunk = blockIdx.x;
    const int layer = item < 12 ? item >> 2 : 3, mt = item < 12 ? item & 3 : 0;
    const int64_t cap = rb.rows;
    const uint16_t *act = rb.act + (int64_t)layer * cap * 64;
    const uint16_t *dz = rb.dz + (int64_t)layer * cap * 64;
    const int ldz = layer < 3 ? 64 : 16;
    const int n0 = 16 * mt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    WgradScratch &S = scr[warp];
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    const int64_t begin = (int64_t)chunk * kWgradChunk;
    const int64_t end = min((int64_t)rows, begin + kWgradChunk);
    for (int64_t r0 = begin + 16 * warp; r0 < end; r0 += 64) {
        {   // gradient tile: 16 rows x 16 columns
            const int rr = lane >> 1, half = lane & 1;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + rr < end) v = *reinterpret_cast<const uint4 *>(dz + (r0 + rr) * ldz + n0 + 8 * half);
            *reinterpret_cast<uint4 *>(S.dzs + rr * 24 + 8 * half) = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // activation tile: 16 rows x 64 columns
            const int idx = lane + 32 * q, rr = idx >> 3, part = idx & 7;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + rr < end) v = *reinterpret_cast<const uint4 *>(act + (r0 + rr) * 64 + 8 * part);
            *reinterpret_cast<uint4 *>(S.as + rr * LDW + 8 * part) = v;
        }
        __syncwarp();
        uint32_t a[4];
        {
            const int q = lane >> 3;
            ldsm_x4_trans(a[0], a[1], a[2], a[3], S.dzs + ((q >> 1) * 8 + (lane & 7)) * 24 + (q & 1) * 8);
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int q = lane >> 3;
            uint32_t b0, b1, b2, b3;
            ldsm_x4_trans(b0, b1, b2, b3, S.as + ((q & 1) * 8 + (lane & 7)) * LDW + 16 * jj + (q >> 1) * 8);
            mma(acc[2 * jj], a, b0, b1);
            mma(acc[2 * jj + 1], a, b2, b3);
        }
        __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[warp][(g + 8 * (e >> 1)) * 64 + 8 * j + 2 * c + (e & 1)] = acc[j][e];
    __syncthreads();
    float *out = partial + ((int64_t)chunk * kWgradItems + item) * 1024;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) out[i] = red[0][i] + red[1][i] + red[2][i] + red[3][i];
}

__global__ void wgrad_reduce_kernel(const float *__restrict__ partial, int n_chunks, float *__restrict__ dW,
                                    const double *__restrict__ loss_part, int n_loss, double *loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kWeights) {
        int item, local;
        if (i < kOffW3) {
            const int layer = i >> 12, r = i & 4095, nn = r >> 6, m = r & 63;
            item = layer * 4 + (nn >> 4);
            local = (nn & 15) * 64 + m;
        } else {
            item = 12;
            local = i - kOffW3;
        }
        float s = 0.0f;
        for (int ch = 0; ch < n_chunks; ++ch) s += partial[((int64_t)ch * kWgradItems + item) * 1024 + local];
        dW[i] = s;
    }
    if (i == 0 && loss) {
        double s = 0.0;
        for (int k = 0; k < n_loss; ++k) s += loss_part[k];
        *loss = s;
    }
}

// ---------------------------------------------------------------------------
// Adam
// ---------------------------------------------------------------------------
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2, uint16_t *__restrict__ bf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        if (bf) bf[i] = bf16_bits(pi);
    }
}

// ---------------------------------------------------------------------------
// encoding of points and texels
// ---------------------------------------------------------------------------
__global__ void encode_points_kernel(const float *__restrict__ xn, int32_t n, const float *__restrict__ table,
                                     float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * kLevels) return;
    const int64_t pt = i / kLevels;
    const int level = (int)(i % kLevels);
    const float x[3] = {xn[3 * pt], xn[3 * pt + 1], xn[3 * pt + 2]};
    const float2 e = encode_level(x, level, table);
    out[pt * 32 + 2 * level] = e.x;
    out[pt * 32 + 2 * level + 1] = e.y;
}

__global__ void encode_texels_kernel(const TexelView tv, const float *__restrict__ table, uint16_t *__restrict__ enc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tv.n_pad * kLevels) return;
    const int64_t t = i / kLevels;
    const int level = (int)(i % kLevels);
    float x[3];
    normalised(tv, tv.pos[t], x);
    const float2 e = encode_level(x, level, table);
    *reinterpret_cast<uint32_t *>(enc + t * 32 + 2 * level) = pack2(e.x, e.y);
}

// ---------------------------------------------------------------------------
// design objective
// ---------------------------------------------------------------------------
__device__ __forceinline__ void design_rows(const DesignArgs &A, WarpScratch *ws, int lane, int l, int64_t t0) {
    if (lane < 16) {
        const int64_t t = t0 + lane;
        const float4 P = A.tex.pos[t], N = A.tex.nrm[t];
        uint16_t *row = ws->X + lane * LDW;
        ws->D[lane] = geometry_row(A.lights[l], P, N, A.tex, row);
        const uint4 *src = reinterpret_cast<const uint4 *>(A.enc + t * 32);
        uint4 *dst = reinterpret_cast<uint4 *>(row);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = src[k];
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kMlpWarps * 32, 2) design_forward_kernel(const DesignArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *sw = reinterpret_cast<uint16_t *>(smem_raw);
    load_weights(sw, A.Wb, false);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    WarpScratch *ws = reinterpret_cast<WarpScratch *>(smem_raw + (size_t)S_FWD_END * 2) + warp;
    const int64_t tpl = A.tex.n_pad / 16;
    const int64_t tiles = tpl * A.n_lights;
    for (int64_t tile = (int64_t)blockIdx.x * kMlpWarps + warp; tile < tiles; tile += (int64_t)gridDim.x * kMlpWarps) {
        const int l = (int)(tile / tpl);
        const int64_t t0 = (tile % tpl) * 16;
        design_rows(A, ws, lane, l, t0);
        uint32_t act[3][4][4];
        float o[2][4];
        forward(sw, ws->X, act, o, g, c);
        if (c == 0)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                const float K = sigmoidf_(o[0][2 * h]) * ws->D[r] + kRScale * softplusf_(o[0][2 * h + 1]);
                A.K[(int64_t)l * A.tex.n_pad + t0 + r] = K;
            }
        __syncwarp();
    }
}

__global__ void design_reduce_kernel(const TexelView tv, const LightC *__restrict__ lights, int32_t n_lights,
                                     const float *__restrict__ K, const float *__restrict__ target,
                                     const float *__restrict__ alpha, float *__restrict__ E_out, float *__restrict__ up,
                                     double *__restrict__ loss_part) {
    __shared__ double red[256];
    double loss = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tv.n_pad; t += (int64_t)gridDim.x * blockDim.x) {
        float E = 0.0f;
        for (int l = 0; l < n_lights; ++l) E += lights[l].intensity * K[(int64_t)l * tv.n_pad + t];
        float u = 0.0f;
        if (t < tv.n) {
            const float d = E - target[t];
            const float w = (alpha ? alpha[t] : 1.0f) * d;
            u = tv.area[t] * w;
            loss += 0.5 * (double)u * (double)d;
            if (E_out) E_out[t] = E;
        }
        up[t] = u;
    }
    red[threadIdx.x] = loss;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kMlpWarps * 32, 2) design_backward_kernel(const DesignArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *sw = reinterpret_cast<uint16_t *>(smem_raw);
    load_weights(sw, A.Wb, true);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    WarpScratch *ws = reinterpret_cast<WarpScratch *>(smem_raw + (size_t)S_ALL_END * 2) + warp;
    const int64_t tpl = A.tex.n_pad / 16;
    const int64_t tiles = tpl * A.n_lights;
    for (int64_t tile = (int64_t)blockIdx.x * kMlpWarps + warp; tile < tiles; tile += (int64_t)gridDim.x * kMlpWarps) {
        const int l = (int)(tile / tpl);
        const int64_t t0 = (tile % tpl) * 16;
        const LightC &L = A.lights[l];
        design_rows(A, ws, lane, l, t0);
        uint32_t act[3][4][4];
        float o[2][4];
        forward(sw, ws->X, act, o, g, c);
        uint32_t dO[4] = {0u, 0u, 0u, 0u};
        if (c == 0)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                const float D = ws->D[r];
                const float v = sigmoidf_(o[0][2 * h]);
                const float K = v * D + kRScale * softplusf_(o[0][2 * h + 1]);
                const float u = A.up[t0 + r];
                const float ui = u * L.intensity;       // dO/dK
                ws->aux0[r] = ui * v;                   // dO/dD
                ws->aux1[r] = u * K;                    // dO/dI
                dO[h] = pack2(ui * v * (1.0f - v) * D, ui * kRScale * sigmoidf_(o[0][2 * h + 1]));
            }
        float dX[8][4];
        backward(sw, act, dO, dX, g, c, nullptr, 0, 0);
        // input entries 32..48 sit in tiles 4..6
#pragma unroll
        for (int j = 4; j < 7; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = 8 * j + 2 * c + (e & 1) - 32;
                if (col < kGeom) ws->gX[g + 8 * (e >> 1)][col] = dX[j][e];
            }
        __syncwarp();
        float gs[7] = {0, 0, 0, 0, 0, 0, 0};
        if (lane < 16) {
            const int64_t t = t0 + lane;
            float gr[6];
            geometry_grad(L, A.tex.pos[t], A.tex.nrm[t], A.tex, ws->gX[lane], ws->aux0[lane], gr);
#pragma unroll
            for (int k = 0; k < 6; ++k) gs[k] = gr[k];
            gs[6] = ws->aux1[lane];
        }
#pragma unroll
        for (int k = 0; k < 7; ++k)
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) gs[k] += __shfl_xor_sync(0xffffffffu, gs[k], off);
        if (lane == 0) {
            float *out = A.gpart + tile * 8;
#pragma unroll
            for (int k = 0; k < 7; ++k) out[k] = gs[k];
            out[7] = 0.0f;
        }
        __syncwarp();
    }
}

__global__ void design_final_kernel(const float *__restrict__ gpart, const LightC *__restrict__ lights,
                                    int32_t n_lights, int64_t tpl, const double *__restrict__ loss_part,
                                    int32_t n_loss_part, double *__restrict__ out) {
    __shared__ double red[7][256];
    const int l = blockIdx.x;
    if (l == n_lights) {   // the objective
        double s = 0.0;
        if (threadIdx.x == 0) {
            for (int k = 0; k < n_loss_part; ++k) s += loss_part[k];
            out[(int64_t)n_lights * 8] = s;
        }
        return;
    }
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = threadIdx.x; i < tpl; i += blockDim.x) {
        const float *p = gpart + ((int64_t)l * tpl + i) * 8;
#pragma unroll
        for (int k = 0; k < 7; ++k) s[k] += (double)p[k];
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
#pragma unroll
            for (int k = 0; k < 7; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *o = out + (int64_t)l * 8;
        o[0] = red[0][0];
        o[1] = red[1][0];
        o[2] = red[2][0];
        o[3] = red[3][0];
        o[4] = red[4][0];
        o[5] = red[6][0] * (double)lights[l].p_int;   // dI/dp_int = p_int
        o[6] = red[5][0];
        o[7] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// The design forward on the 5th-generation tensor cores (tcgen05)
//
// A warpgroup of 128 threads takes 128 rows at a time, one row per thread.
// The thread writes its input row into shared memory in the canonical
// no-swizzle K-major layout (8 x 8 bf16 "core matrices" of 128 bytes; core
// (r / 8, k / 8) at ((r / 8) * 8 + k / 8) * 128 bytes), one elected thread
// issues the four K = 16 steps of each layer as tcgen05.mma (M = 128,
// N = 64 or 16, bf16 x bf16 -> fp32 in tensor memory) and commits them to an
// mbarrier; every thread then reads its accumulator row back with
// tcgen05.ld, applies ReLU, rounds to bf16 and writes the next layer's
// operand. A CTA holds kTcTiles such warpgroups, each with its own operand
// tile, 64 TMEM columns, mbarrier and named barrier, so their tiles proceed
// independently (one's MMA overlaps another's epilogue) while they share one
// copy of the weights, stored in the same layout and loaded once per CTA.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr int kTcTiles = 4;                      // warpgroups (128-row tiles) per CTA
constexpr int kTcThreads = kTcRows * kTcTiles;
constexpr uint32_t kTcCols = 64;                 // TMEM columns of one 128 x 64 fp32 accumulator
constexpr uint32_t kTcSpin = 1u << 20;           // mbarrier polls before giving up
constexpr int kErrTc = 1;

struct alignas(1024) TcSmem {
    uint16_t a[kTcTiles][kTcRows * 64];          // A operand of each warpgroup, 16 KB each
    uint16_t w[3 * 64 * 64 + 16 * 64];           // B operands, layer after layer
    unsigned long long mbar[kTcTiles];
    uint32_t tmem;
    int32_t abort[kTcTiles];                     // set and read by one warpgroup only
};

// Two CTAs fit an SM's 228 KB of shared memory and a third does not, so the
// 2 x kTcTiles x 64 TMEM columns of the resident CTAs never exceed 512.
static_assert(2 * (sizeof(TcSmem) + 2048) <= 228 * 1024 && 3 * (sizeof(TcSmem) + 1024) > 228 * 1024,
              "design forward: exactly two CTAs per SM");
static_assert(2 * kTcCols * kTcTiles <= 512, "TMEM columns of two CTAs");

// Barrier of the 128 threads of warpgroup g (named barrier 1 + g; barrier 0
// is __syncthreads).
__device__ __forceinline__ void wg_sync(int g) { asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g) : "memory"); }

__device__ __forceinline__ uint32_t core_offset(int r, int k) {      // bytes, 64-wide rows
    return (uint32_t)((((r >> 3) << 3) + (k >> 3)) << 7) + (uint32_t)((r & 7) << 4) + (uint32_t)((k & 7) << 1);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset
// (between core matrices adjacent in K), stride byte offset (between core
// matrices adjacent in M / N), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (uint32_t i = 0; i < kTcSpin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// After a warpgroup gave up waiting (its flag set): wait once more, with a
// limit eight times as long, for the commit it gave up on, so that no MMA of
// its own is still writing tensor memory when the CTA frees it. If that wait
// gives up too, the memory is freed all the same (the kernel has already
// reported the error).
__device__ __forceinline__ void tc_drain(uint32_t mbar, uint32_t pending_phase) {
    for (int i = 0; i < 8; ++i)
        if (mbar_wait(mbar, pending_phase)) return;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 16 fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 2) design_forward_tc_kernel(const DesignArgs A, int32_t *err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_raw);
    const int tid = threadIdx.x, warp = tid >> 5, g = tid / kTcRows, r = tid % kTcRows;
    // weights into the canonical layout
    for (int i = tid; i < kWeights; i += kTcThreads) {
        const int layer = i < kOffW3 ? i >> 12 : 3, q = i < kOffW3 ? i & 4095 : i - kOffW3;
        const int n = q >> 6, k = q & 63;
        *reinterpret_cast<uint16_t *>(reinterpret_cast<unsigned char *>(S.w) + layer * 8192 + core_offset(n, k)) =
            A.Wb[i];
    }
    if (tid == 0) {
        for (int k = 0; k < kTcTiles; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&S.mbar[k])) : "memory");
            S.abort[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTcCols * kTcTiles)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // this warpgroup's accumulator columns; a warp reads TMEM lanes 32 (warp % 4) ..
    const uint32_t tmem = S.tmem + (uint32_t)g * kTcCols;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t mbar = smem_u32(&S.mbar[g]);
    const uint32_t a_base = smem_u32(S.a[g]), w_base = smem_u32(S.w);
    const int64_t rows = A.tex.n_pad * (int64_t)A.n_lights;
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    uint32_t phase = 0;
    unsigned char *arow = reinterpret_cast<unsigned char *>(S.a[g]);
    for (int64_t tile = (int64_t)blockIdx.x * kTcTiles + g; tile < tiles; tile += (int64_t)gridDim.x * kTcTiles) {
        const int64_t row = tile * kTcRows + r;
        const bool valid = row < rows;
        const int l = valid ? (int)(row / A.tex.n_pad) : 0;
        const int64_t t = valid ? row % A.tex.n_pad : 0;
        // the input row: encoding (cached per texel) and geometric features
        uint16_t x[64];
        const float D = geometry_row(A.lights[l], A.tex.pos[t], A.tex.nrm[t], A.tex, x);
        const uint4 *enc = reinterpret_cast<const uint4 *>(A.enc + t * 32);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8)
            *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = valid ? enc[g8] : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int g8 = 4; g8 < 8; ++g8) {
            uint4 v;
            v.x = valid ? (uint32_t)x[8 * g8] | ((uint32_t)x[8 * g8 + 1] << 16) : 0u;
            v.y = valid ? (uint32_t)x[8 * g8 + 2] | ((uint32_t)x[8 * g8 + 3] << 16) : 0u;
            v.z = valid ? (uint32_t)x[8 * g8 + 4] | ((uint32_t)x[8 * g8 + 5] << 16) : 0u;
            v.w = valid ? (uint32_t)x[8 * g8 + 6] | ((uint32_t)x[8 * g8 + 7] << 16) : 0u;
            *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = v;
        }
        proxy_fence();
        wg_sync(g);
        float o0 = 0.0f, o1 = 0.0f;
        for (int layer = 0; layer < 4; ++layer) {
            const int N = layer < 3 ? 64 : 16;
            if (r == 0) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem, smem_desc(a_base + 256 * kk, 128, 1024),
                           smem_desc(w_base + layer * 8192 + 256 * kk, 128, 1024), mma_idesc(128, N), kk > 0);
                tc_commit(mbar);
            }
            const bool ok = mbar_wait(mbar, phase);
            phase ^= 1u;
            tc_fence_after();
            if (!ok) S.abort[g] = 1;
            wg_sync(g);
            if (S.abort[g]) break;
            if (layer < 3) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint4 q;
                        q.x = pack2(fmaxf(v[8 * h], 0.0f), fmaxf(v[8 * h + 1], 0.0f));
                        q.y = pack2(fmaxf(v[8 * h + 2], 0.0f), fmaxf(v[8 * h + 3], 0.0f));
                        q.z = pack2(fmaxf(v[8 * h + 4], 0.0f), fmaxf(v[8 * h + 5], 0.0f));
                        q.w = pack2(fmaxf(v[8 * h + 6], 0.0f), fmaxf(v[8 * h + 7], 0.0f));
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, 16 * c + 8 * h)) = q;
                    }
                }
                tc_fence_before();
                proxy_fence();
                wg_sync(g);
            } else {
                float v[16];
                tc_ld16(lane_addr, v);
                o0 = v[0];
                o1 = v[1];
                tc_fence_before();
            }
        }
        if (S.abort[g]) break;
        if (valid) A.K[row] = sigmoidf_(o0) * D + kRScale * softplusf_(o1);
        wg_sync(g);
    }
    if (S.abort[g]) tc_drain(mbar, phase ^ 1u);      // the commit given up on is the pending phase
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        int32_t any = 0;
        for (int k = 0; k < kTcTiles; ++k) any |= S.abort[k];
        if (any) atomicOr(err, kErrTc);
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(S.tmem), "r"(kTcCols * kTcTiles)
                     : "memory");
}

// The design backward on tcgen05: per 128-row tile the forward again (ReLU
// masks kept as bits), the loss head, then the gradient through W3^T, W2^T,
// W1^T, W0^T as tcgen05.mma on transposed weights (the output layer's step
// has K = 16), and each thread's row through the feature Jacobian.
template <int kTiles>
struct alignas(1024) TcBwdSmemT {
    uint16_t a[kTiles][kTcRows * 64];            // per warpgroup: activations, then gradients (64 wide)
    uint16_t d4[kTiles][kTcRows * 16];           // per warpgroup: gradient at the outputs (16 wide)
    uint16_t w[3 * 64 * 64 + 16 * 64];           // W0, W1, W2 [64][64], W3 [16][64]
    uint16_t wt[3 * 64 * 64 + 64 * 16];          // W0^T, W1^T, W2^T [64][64], W3^T [64][16]
    unsigned long long mbar[kTiles];
    double red[2 * kTiles * kTcRows / 32];       // per-warp loss sums (training: two threads per row)
    uint32_t tmem;
    int32_t abort[kTiles];                       // set and read by one warpgroup only
};
using TcBwdSmem = TcBwdSmemT<kTcTiles>;

// One CTA per SM (shared memory admits no second): kTcTiles x 64 TMEM columns.
static_assert(sizeof(TcBwdSmem) + 1024 <= 227 * 1024 && 2 * (sizeof(TcBwdSmem) + 1024) > 228 * 1024,
              "design backward: exactly one CTA per SM");

// The training kernel's 128-row tiles per CTA (a build knob), each carried by
// two threads per row (256 threads: warps w and w + 4 of a tile read the same
// TMEM lanes, columns 0..31 and 32..63), its TMEM allocation (a power of
// two), and the guarantee that the CTAs resident on an SM never ask for more
// than 512 columns.
#ifndef SG_TRAIN_TILES
#define SG_TRAIN_TILES 2
#endif
constexpr int kTrainTiles = SG_TRAIN_TILES;
constexpr int kTrainTileThreads = 2 * kTcRows;
constexpr int kTrainThreads = kTrainTiles * kTrainTileThreads;
using TcTrainSmem = TcBwdSmemT<kTrainTiles>;
constexpr uint32_t pow2_cols(uint32_t c) { return c <= 32 ? 32 : (c <= 64 ? 64 : (c <= 128 ? 128 : (c <= 256 ? 256 : 512))); }
constexpr uint32_t kTrainCols = pow2_cols(kTcCols * kTrainTiles);
static_assert(kTrainTiles >= 1 && kTcCols * kTrainTiles <= 512, "training tiles fit TMEM");
static_assert(sizeof(TcTrainSmem) + 1024 <= 227 * 1024, "training CTA fits shared memory");
constexpr int kTrainCtasPerSm = (int)((228 * 1024) / (sizeof(TcTrainSmem) + 2048));
#ifndef SG_TRAIN_MIN_CTAS
#define SG_TRAIN_MIN_CTAS 2
#endif
constexpr int kTrainMinCtas = SG_TRAIN_MIN_CTAS;   // register budget: 65536 / (threads x this)
static_assert(kTrainCtasPerSm >= 1 && kTrainCtasPerSm * kTrainCols <= 512,
              "resident training CTAs never exceed 512 TMEM columns");

__device__ __forceinline__ uint32_t core_offset16(int r, int k) {    // bytes, 16-wide rows
    return (uint32_t)((((r >> 3) << 1) + (k >> 3)) << 7) + (uint32_t)((r & 7) << 4) + (uint32_t)((k & 7) << 1);
}

// W and W^T into the canonical layouts (W3^T is 64 x 16: 16-wide rows).
template <class Smem>
__device__ __forceinline__ void stage_weights_bwd(Smem &S, const uint16_t *__restrict__ Wb, int tid, int nthreads) {
    unsigned char *wb = reinterpret_cast<unsigned char *>(S.w), *wtb = reinterpret_cast<unsigned char *>(S.wt);
    for (int i = tid; i < kWeights; i += nthreads) {
        const uint16_t v = Wb[i];
        if (i < kOffW3) {
            const int layer = i >> 12, r = i & 4095, n = r >> 6, k = r & 63;
            *reinterpret_cast<uint16_t *>(wb + layer * 8192 + core_offset(n, k)) = v;
            *reinterpret_cast<uint16_t *>(wtb + layer * 8192 + core_offset(k, n)) = v;
        } else {
            const int r = i - kOffW3, n = r >> 6, k = r & 63;        // W3[n][k], n < 16
            *reinterpret_cast<uint16_t *>(wb + 3 * 8192 + core_offset(n, k)) = v;
            *reinterpret_cast<uint16_t *>(wtb + 3 * 8192 + core_offset16(k, n)) = v;
        }
    }
}

// Issues one layer (K / 16 steps) from thread r == 0 of the warpgroup and
// waits for it; false if the wait gave up.
__device__ __forceinline__ bool tc_layer(uint32_t tmem, uint32_t a, uint32_t a_sbo, uint32_t b, uint32_t b_sbo, int N,
                                         int ksteps, uint32_t mbar, uint32_t &phase, int r) {
    if (r == 0) {
        tc_fence_after();
        for (int kk = 0; kk < ksteps; ++kk)
            tc_mma(tmem, smem_desc(a + 256 * kk, 128, a_sbo), smem_desc(b + 256 * kk, 128, b_sbo), mma_idesc(128, N),
                   kk > 0);
        tc_commit(mbar);
    }
    const bool ok = mbar_wait(mbar, phase);
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

__global__ void __launch_bounds__(kTcThreads, 1) design_backward_tc_kernel(const DesignArgs A, int32_t *err) {
    extern __shared__ __align__(1024) unsigned char tcb_raw[];
    TcBwdSmem &S = *reinterpret_cast<TcBwdSmem *>(tcb_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = tid / kTcRows, r = tid % kTcRows;
    stage_weights_bwd(S, A.Wb, tid, kTcThreads);
    if (tid == 0) {
        for (int k = 0; k < kTcTiles; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&S.mbar[k])) : "memory");
            S.abort[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTcCols * kTcTiles)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem + (uint32_t)g * kTcCols;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t mbar = smem_u32(&S.mbar[g]);
    const uint32_t a_addr = smem_u32(S.a[g]), d4_addr = smem_u32(S.d4[g]), w_addr = smem_u32(S.w),
                   wt_addr = smem_u32(S.wt);
    const int64_t rows = A.tex.n_pad * (int64_t)A.n_lights;
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    uint32_t phase = 0;
    unsigned char *arow = reinterpret_cast<unsigned char *>(S.a[g]), *drow = reinterpret_cast<unsigned char *>(S.d4[g]);
    for (int64_t tile = (int64_t)blockIdx.x * kTcTiles + g; tile < tiles; tile += (int64_t)gridDim.x * kTcTiles) {
        const int64_t row = tile * kTcRows + r;
        const bool valid = row < rows;
        const int l = valid ? (int)(row / A.tex.n_pad) : 0;
        const int64_t t = valid ? row % A.tex.n_pad : 0;
        const LightC &L = A.lights[l];
        const float4 P = A.tex.pos[t], Nt = A.tex.nrm[t];
        uint16_t x[64];
        const float D = geometry_row(L, P, Nt, A.tex, x);
        const uint4 *enc = reinterpret_cast<const uint4 *>(A.enc + t * 32);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8)
            *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = valid ? enc[g8] : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int g8 = 4; g8 < 8; ++g8) {
            uint4 v;
            v.x = valid ? (uint32_t)x[8 * g8] | ((uint32_t)x[8 * g8 + 1] << 16) : 0u;
            v.y = valid ? (uint32_t)x[8 * g8 + 2] | ((uint32_t)x[8 * g8 + 3] << 16) : 0u;
            v.z = valid ? (uint32_t)x[8 * g8 + 4] | ((uint32_t)x[8 * g8 + 5] << 16) : 0u;
            v.w = valid ? (uint32_t)x[8 * g8 + 6] | ((uint32_t)x[8 * g8 + 7] << 16) : 0u;
            *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = v;
        }
        proxy_fence();
        wg_sync(g);
        uint32_t mask[3][2];
        float o0 = 0.0f, o1 = 0.0f;
        bool ok = true;
        // forward
        for (int layer = 0; layer < 4 && ok; ++layer) {
            const int N = layer < 3 ? 64 : 16;
            ok = tc_layer(tmem, a_addr, 1024, w_addr + layer * 8192, 1024, N, 4, mbar, phase, r);
            if (!ok) S.abort[g] = 1;
            wg_sync(g);
            if (S.abort[g]) { ok = false; break; }
            if (layer < 3) {
                mask[layer][0] = mask[layer][1] = 0u;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (v[i] > 0.0f) mask[layer][c >> 1] |= 1u << ((c & 1) * 16 + i);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint4 q;
                        q.x = pack2(fmaxf(v[8 * h], 0.0f), fmaxf(v[8 * h + 1], 0.0f));
                        q.y = pack2(fmaxf(v[8 * h + 2], 0.0f), fmaxf(v[8 * h + 3], 0.0f));
                        q.z = pack2(fmaxf(v[8 * h + 4], 0.0f), fmaxf(v[8 * h + 5], 0.0f));
                        q.w = pack2(fmaxf(v[8 * h + 6], 0.0f), fmaxf(v[8 * h + 7], 0.0f));
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, 16 * c + 8 * h)) = q;
                    }
                }
            } else {
                float v[16];
                tc_ld16(lane_addr, v);
                o0 = v[0];
                o1 = v[1];
            }
            tc_fence_before();
            proxy_fence();
            wg_sync(g);
        }
        if (!ok) break;
        // loss head: dO/do of the row
        const float sg0 = sigmoidf_(o0);
        const float K = sg0 * D + kRScale * softplusf_(o1);
        const float u = valid ? A.up[t] : 0.0f;
        const float ui = u * L.intensity;
        const float gD = ui * sg0, gI = u * K;
        {
            uint4 q0, q1 = make_uint4(0, 0, 0, 0);
            q0.x = pack2(ui * sg0 * (1.0f - sg0) * D, ui * kRScale * sigmoidf_(o1));
            q0.y = q0.z = q0.w = 0u;
            *reinterpret_cast<uint4 *>(drow + core_offset16(r, 0)) = q0;
            *reinterpret_cast<uint4 *>(drow + core_offset16(r, 8)) = q1;
        }
        proxy_fence();
        wg_sync(g);
        // backward: W3^T (K = 16), then W2^T, W1^T (masked, rounded), W0^T
        float gX[kGeom];
        for (int layer = 3; layer >= 0 && ok; --layer) {
            if (layer == 3) ok = tc_layer(tmem, d4_addr, 256, wt_addr + 3 * 8192, 256, 64, 1, mbar, phase, r);
            else ok = tc_layer(tmem, a_addr, 1024, wt_addr + layer * 8192, 1024, 64, 4, mbar, phase, r);
            if (!ok) S.abort[g] = 1;
            wg_sync(g);
            if (S.abort[g]) { ok = false; break; }
            if (layer > 0) {
                const int m = layer - 1;          // the mask of the product's input
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float z[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int col = 16 * c + 8 * h + i;
                            z[i] = (mask[m][col >> 5] >> (col & 31)) & 1u ? v[8 * h + i] : 0.0f;
                        }
                        uint4 q;
                        q.x = pack2(z[0], z[1]);
                        q.y = pack2(z[2], z[3]);
                        q.z = pack2(z[4], z[5]);
                        q.w = pack2(z[6], z[7]);
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, 16 * c + 8 * h)) = q;
                    }
                }
            } else {
                float v[16];
                tc_ld16(lane_addr + 32, v);       // input entries 32..47
#pragma unroll
                for (int i = 0; i < 16; ++i) gX[i] = v[i];
                tc_ld16(lane_addr + 48, v);       // 48..63
                gX[16] = v[0];
            }
            tc_fence_before();
            proxy_fence();
            wg_sync(g);
        }
        if (!ok) break;
        float gs[7] = {0, 0, 0, 0, 0, 0, 0};
        if (valid) {
            float gr[6];
            geometry_grad(L, P, Nt, A.tex, gX, gD, gr);
#pragma unroll
            for (int k = 0; k < 6; ++k) gs[k] = gr[k];
            gs[6] = gI;
        }
#pragma unroll
        for (int k = 0; k < 7; ++k)
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) gs[k] += __shfl_xor_sync(0xffffffffu, gs[k], off);
        if ((lane & 15) == 0 && valid) {
            float *out = A.gpart + (row / 16) * 8;
#pragma unroll
            for (int k = 0; k < 7; ++k) out[k] = gs[k];
            out[7] = 0.0f;
        }
    }
    if (S.abort[g]) tc_drain(mbar, phase ^ 1u);      // the commit given up on is the pending phase
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        int32_t any = 0;
        for (int k = 0; k < kTcTiles; ++k) any |= S.abort[k];
        if (any) atomicOr(err, kErrTc);
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(S.tmem), "r"(kTcCols * kTcTiles)
                     : "memory");
}

// The design objective in one kernel for up to kFusedMaxLights lights: a
// 128-row tile holds all lights of 128 / n texels (row = texel x n + light),
// so after the forward the tile forms each texel's irradiance E_t (the sum
// over its rows in light order), the objective's share and the weight
// u_t = A_t alpha_t (E_t - E*_t) itself, and goes straight into the backward
// without recomputing the forward; the per-light gradient sums over the
// tile's texels go to gpart[light][tile].
__global__ void __launch_bounds__(kTcThreads, 1) design_fused_tc_kernel(const DesignArgs A, const FusedArgs F,
                                                                       int32_t *err) {
    extern __shared__ __align__(1024) unsigned char tcb_raw[];
    TcBwdSmem &S = *reinterpret_cast<TcBwdSmem *>(tcb_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = tid / kTcRows, r = tid % kTcRows;
    stage_weights_bwd(S, A.Wb, tid, kTcThreads);
    if (tid == 0) {
        for (int k = 0; k < kTcTiles; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&S.mbar[k])) : "memory");
            S.abort[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTcCols * kTcTiles)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem + (uint32_t)g * kTcCols;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t mbar = smem_u32(&S.mbar[g]);
    const uint32_t a_addr = smem_u32(S.a[g]), d4_addr = smem_u32(S.d4[g]), w_addr = smem_u32(S.w),
                   wt_addr = smem_u32(S.wt);
    const int nl = A.n_lights, tpt = F.texels_per_tile;
    const int tl = r / nl, l_row = r % nl;                  // this row: texel tl of the tile, light l_row
    uint32_t phase = 0;
    double loss = 0.0;
    float *scr = reinterpret_cast<float *>(S.a[g]);         // free between the forward and the backward
    float *gsum = reinterpret_cast<float *>(S.d4[g]);       // free after the backward's first product
    unsigned char *arow = reinterpret_cast<unsigned char *>(S.a[g]), *drow = reinterpret_cast<unsigned char *>(S.d4[g]);
    for (int64_t tile = (int64_t)blockIdx.x * kTcTiles + g; tile < F.n_tiles; tile += (int64_t)gridDim.x * kTcTiles) {
        const int64_t tt = tile * tpt + tl;
        const bool valid = tl < tpt && tt < A.tex.n_pad;
        const int l = valid ? l_row : 0;
        const int64_t t = valid ? tt : 0;
        const LightC &L = A.lights[l];
        const float4 P = A.tex.pos[t], Nt = A.tex.nrm[t];
        uint16_t x[64];
        const float D = geometry_row(L, P, Nt, A.tex, x);
        const uint4 *enc = reinterpret_cast<const uint4 *>(A.enc + t * 32);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8)
            *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = valid ? enc[g8] : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int g8 = 4; g8 < 8; ++g8) {
            uint4 v;
            v.x = valid ? (uint32_t)x[8 * g8] | ((uint32_t)x[8 * g8 + 1] << 16) : 0u;
            v.y = valid ? (uint32_t)x[8 * g8 + 2] | ((uint32_t)x[8 * g8 + 3] << 16) : 0u;
            v.z = valid ? (uint32_t)x[8 * g8 + 4] | ((uint32_t)x[8 * g8 + 5] << 16) : 0u;
            v.w = valid ? (uint32_t)x[8 * g8 + 6] | ((uint32_t)x[8 * g8 + 7] << 16) : 0u;
            *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = v;
        }
        proxy_fence();
        wg_sync(g);
        uint32_t mask[3][2];
        float o0 = 0.0f, o1 = 0.0f;
        bool ok = true;
        // forward
        for (int layer = 0; layer < 4 && ok; ++layer) {
            const int N = layer < 3 ? 64 : 16;
            ok = tc_layer(tmem, a_addr, 1024, w_addr + layer * 8192, 1024, N, 4, mbar, phase, r);
            if (!ok) S.abort[g] = 1;
            wg_sync(g);
            if (S.abort[g]) { ok = false; break; }
            if (layer < 3) {
                mask[layer][0] = mask[layer][1] = 0u;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (v[i] > 0.0f) mask[layer][c >> 1] |= 1u << ((c & 1) * 16 + i);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint4 q;
                        q.x = pack2(fmaxf(v[8 * h], 0.0f), fmaxf(v[8 * h + 1], 0.0f));
                        q.y = pack2(fmaxf(v[8 * h + 2], 0.0f), fmaxf(v[8 * h + 3], 0.0f));
                        q.z = pack2(fmaxf(v[8 * h + 4], 0.0f), fmaxf(v[8 * h + 5], 0.0f));
                        q.w = pack2(fmaxf(v[8 * h + 6], 0.0f), fmaxf(v[8 * h + 7], 0.0f));
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, 16 * c + 8 * h)) = q;
                    }
                }
            } else {
                float v[16];
                tc_ld16(lane_addr, v);
                o0 = v[0];
                o1 = v[1];
            }
            tc_fence_before();
            proxy_fence();
            wg_sync(g);
        }
        if (!ok) break;
        // loss head: dO/do of the row
        const float sg0 = sigmoidf_(o0);
        const float K = sg0 * D + kRScale * softplusf_(o1);
        // the texel's irradiance E_t = sum_l I_l K(t, l), summed in light order
        scr[r] = valid ? L.intensity * K : 0.0f;
        wg_sync(g);
        float u = 0.0f;
        if (valid) {
            float E = 0.0f;
            for (int q = 0; q < nl; ++q) E += scr[tl * nl + q];
            if (t < A.tex.n) {
                const float d = E - F.target[t];
                const float w = (F.alpha ? F.alpha[t] : 1.0f) * d;
                u = A.tex.area[t] * w;
                if (l == 0) {
                    loss += 0.5 * (double)u * (double)d;
                    if (F.E_out) F.E_out[t] = E;
                }
            }
        }
        const float ui = u * L.intensity;
        const float gD = ui * sg0, gI = u * K;
        {
            uint4 q0, q1 = make_uint4(0, 0, 0, 0);
            q0.x = pack2(ui * sg0 * (1.0f - sg0) * D, ui * kRScale * sigmoidf_(o1));
            q0.y = q0.z = q0.w = 0u;
            *reinterpret_cast<uint4 *>(drow + core_offset16(r, 0)) = q0;
            *reinterpret_cast<uint4 *>(drow + core_offset16(r, 8)) = q1;
        }
        proxy_fence();
        wg_sync(g);
        // backward: W3^T (K = 16), then W2^T, W1^T (masked, rounded), W0^T
        float gX[kGeom];
        for (int layer = 3; layer >= 0 && ok; --layer) {
            if (layer == 3) ok = tc_layer(tmem, d4_addr, 256, wt_addr + 3 * 8192, 256, 64, 1, mbar, phase, r);
            else ok = tc_layer(tmem, a_addr, 1024, wt_addr + layer * 8192, 1024, 64, 4, mbar, phase, r);
            if (!ok) S.abort[g] = 1;
            wg_sync(g);
            if (S.abort[g]) { ok = false; break; }
            if (layer > 0) {
                const int m = layer - 1;          // the mask of the product's input
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float z[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int col = 16 * c + 8 * h + i;
                            z[i] = (mask[m][col >> 5] >> (col & 31)) & 1u ? v[8 * h + i] : 0.0f;
                        }
                        uint4 q;
                        q.x = pack2(z[0], z[1]);
                        q.y = pack2(z[2], z[3]);
                        q.z = pack2(z[4], z[5]);
                        q.w = pack2(z[6], z[7]);
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, 16 * c + 8 * h)) = q;
                    }
                }
            } else {
                float v[16];
                tc_ld16(lane_addr + 32, v);       // input entries 32..47
#pragma unroll
                for (int i = 0; i < 16; ++i) gX[i] = v[i];
                tc_ld16(lane_addr + 48, v);       // 48..63
                gX[16] = v[0];
            }
            tc_fence_before();
            proxy_fence();
            wg_sync(g);
        }
        if (!ok) break;
        float gs[7] = {0, 0, 0, 0, 0, 0, 0};
        if (valid) {
            float gr[6];
            geometry_grad(L, P, Nt, A.tex, gX, gD, gr);
#pragma unroll
            for (int k = 0; k < 6; ++k) gs[k] = gr[k];
            gs[6] = gI;
        }
        // per-light sums over the tile's texels, in texel order
#pragma unroll
        for (int k = 0; k < 7; ++k) gsum[r * 8 + k] = gs[k];
        wg_sync(g);
        if (r < nl) {
            float acc[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int q = 0; q < tpt; ++q)
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[k] += gsum[(q * nl + r) * 8 + k];
            float *out = A.gpart + ((int64_t)r * F.n_tiles + tile) * 8;
#pragma unroll
            for (int k = 0; k < 7; ++k) out[k] = acc[k];
            out[7] = 0.0f;
        }
        wg_sync(g);
    }
    loss = warp_sum_d(loss);
    if (lane == 0) S.red[warp] = loss;
    if (S.abort[g]) tc_drain(mbar, phase ^ 1u);      // the commit given up on is the pending phase
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < kTcThreads / 32; ++w) sum += S.red[w];
        F.loss_part[blockIdx.x] = sum;
        int32_t any = 0;
        for (int k = 0; k < kTcTiles; ++k) any |= S.abort[k];
        if (any) atomicOr(err, kErrTc);
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(S.tmem), "r"(kTcCols * kTcTiles)
                     : "memory");
}

// The training step's network on tcgen05: per 128-row tile of samples the
// input rows (hash encoding and geometric features), the forward with the
// ReLU masks kept as bits, the loss head, the backward through W3^T .. W0^T
// and the encoding gradient scattered into the table with float2 atomics.
// Two threads carry a row: the first builds the geometric features, encodes
// levels 0..7 and runs the loss head, the second encodes levels 8..15; each
// handles half of the row's 64 accumulator columns in every epilogue and
// scatters the gradient of its own levels. The samples, the loss and the bf16
// rows kept for the weight gradient are those of train_kernel (the same row
// buffers), so wgrad_kernel serves both.
__device__ __forceinline__ void tile_sync(int g) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "r"(kTrainTileThreads) : "memory");
}

__global__ void __launch_bounds__(kTrainThreads, kTrainMinCtas) train_tc_kernel(const TrainArgs A, int32_t *err) {
    extern __shared__ __align__(1024) unsigned char tct_raw[];
    TcTrainSmem &S = *reinterpret_cast<TcTrainSmem *>(tct_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid / kTrainTileThreads, u = tid % kTrainTileThreads;
    const int wt = u >> 5, hf = wt >> 2, r = (wt & 3) * 32 + lane;   // tile warp, column half, row
    stage_weights_bwd(S, A.Wb, tid, kTrainThreads);
    if (tid == 0) {
        for (int k = 0; k < kTrainTiles; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&S.mbar[k])) : "memory");
            S.abort[k] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTrainCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem + (uint32_t)g * kTcCols;
    // TMEM lanes 32 (warp % 4) .. of this tile's columns, this thread's half
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(32 * hf);
    const uint32_t mbar = smem_u32(&S.mbar[g]);
    const uint32_t a_addr = smem_u32(S.a[g]), d4_addr = smem_u32(S.d4[g]), w_addr = smem_u32(S.w),
                   wt_addr = smem_u32(S.wt);
    unsigned char *arow = reinterpret_cast<unsigned char *>(S.a[g]), *drow = reinterpret_cast<unsigned char *>(S.d4[g]);
    const int64_t n = A.tex.n, cap = A.rb.rows;
    const int64_t tiles = ((int64_t)A.batch + kTcRows - 1) / kTcRows;
    const double inv_b = 1.0 / (double)A.batch;
    uint32_t phase = 0;
    double loss = 0.0;
    for (int64_t tile = (int64_t)blockIdx.x * kTrainTiles + g; tile < tiles; tile += (int64_t)gridDim.x * kTrainTiles) {
        const int64_t i = tile * kTcRows + r;
        const bool valid = i < A.batch;
        int32_t smp = 0, t = 0;
        if (valid) {
            if (A.samples) {
                smp = A.samples[2 * i];
                t = A.samples[2 * i + 1];
            } else {
                const uint64_t h = mix64(A.seed ^ mix64((A.step << 32) ^ (uint64_t)i));
                smp = (int32_t)(((h >> 32) * (uint64_t)A.n_solves) >> 32);
                t = (int32_t)(((h & 0xFFFFFFFFull) * (uint64_t)n) >> 32);
            }
        }
        const float4 P = A.tex.pos[t];
        float xn[3];
        normalised(A.tex, P, xn);
        uint16_t *kept = A.rb.act + i * 64;              // this row of the first product's input
        // this thread's levels: entries 16 hf .. 16 hf + 15 of the row
        {
            uint32_t enc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 e = encode_level(xn, 8 * hf + q, A.table);
                enc[q] = pack2(e.x, e.y);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const uint4 v = valid ? make_uint4(enc[4 * q], enc[4 * q + 1], enc[4 * q + 2], enc[4 * q + 3])
                                      : make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4 *>(arow + core_offset(r, 16 * hf + 8 * q)) = v;
                if (valid) *reinterpret_cast<uint4 *>(kept + 16 * hf + 8 * q) = v;
            }
        }
        float D = 0.0f;
        if (hf == 0) {   // geometric features, entries 32..63
            uint16_t x[64];
            D = geometry_row(A.lights[smp], P, A.tex.nrm[t], A.tex, x);
#pragma unroll
            for (int g8 = 4; g8 < 8; ++g8) {
                uint4 v;
                v.x = valid ? (uint32_t)x[8 * g8] | ((uint32_t)x[8 * g8 + 1] << 16) : 0u;
                v.y = valid ? (uint32_t)x[8 * g8 + 2] | ((uint32_t)x[8 * g8 + 3] << 16) : 0u;
                v.z = valid ? (uint32_t)x[8 * g8 + 4] | ((uint32_t)x[8 * g8 + 5] << 16) : 0u;
                v.w = valid ? (uint32_t)x[8 * g8 + 6] | ((uint32_t)x[8 * g8 + 7] << 16) : 0u;
                *reinterpret_cast<uint4 *>(arow + core_offset(r, 8 * g8)) = v;
                if (valid) *reinterpret_cast<uint4 *>(kept + 8 * g8) = v;
            }
        }
        proxy_fence();
        tile_sync(g);
        uint32_t mask[3];
        float o0 = 0.0f, o1 = 0.0f;
        bool ok = true;
        // forward; the activations are also kept as the inputs of products 1..3
        for (int layer = 0; layer < 4 && ok; ++layer) {
            const int N = layer < 3 ? 64 : 16;
            ok = tc_layer(tmem, a_addr, 1024, w_addr + layer * 8192, 1024, N, 4, mbar, phase, u);
            if (!ok) S.abort[g] = 1;
            tile_sync(g);
            if (S.abort[g]) { ok = false; break; }
            if (layer < 3) {
                uint16_t *kl = A.rb.act + (int64_t)(layer + 1) * cap * 64 + i * 64;
                mask[layer] = 0u;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (v[k] > 0.0f) mask[layer] |= 1u << (16 * c + k);
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        uint4 q;
                        q.x = pack2(fmaxf(v[8 * hh], 0.0f), fmaxf(v[8 * hh + 1], 0.0f));
                        q.y = pack2(fmaxf(v[8 * hh + 2], 0.0f), fmaxf(v[8 * hh + 3], 0.0f));
                        q.z = pack2(fmaxf(v[8 * hh + 4], 0.0f), fmaxf(v[8 * hh + 5], 0.0f));
                        q.w = pack2(fmaxf(v[8 * hh + 6], 0.0f), fmaxf(v[8 * hh + 7], 0.0f));
                        const int col = 32 * hf + 16 * c + 8 * hh;
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, col)) = q;
                        if (valid) *reinterpret_cast<uint4 *>(kl + col) = q;
                    }
                }
            } else if (hf == 0) {
                float v[16];
                tc_ld16(lane_addr, v);
                o0 = v[0];
                o1 = v[1];
            }
            tc_fence_before();
            proxy_fence();
            tile_sync(g);
        }
        if (!ok) break;
        // loss head: weighted squared error of K against the solve's irradiance
        if (hf == 0) {
            const float sv = sigmoidf_(o0), sp = softplusf_(o1);
            const float K = sv * D + kRScale * sp;
            const float Eo = valid ? __ldg(A.E_obs + (int64_t)smp * n + t) : 0.0f;
            const float wgt = valid ? A.tex.area[t] * A.tex.inv_mean_area : 0.0f;
            const float e = K - Eo;
            loss += 0.5 * (double)wgt * (double)e * (double)e * inv_b;
            const float dK = (float)((double)(wgt * e) * inv_b);
            const uint4 q0 = make_uint4(pack2(dK * sv * (1.0f - sv) * D, dK * kRScale * sigmoidf_(o1)), 0u, 0u, 0u);
            const uint4 q1 = make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4 *>(drow + core_offset16(r, 0)) = q0;
            *reinterpret_cast<uint4 *>(drow + core_offset16(r, 8)) = q1;
            if (valid) {
                uint16_t *kd = A.rb.dz + 3 * cap * 64 + i * 16;
                *reinterpret_cast<uint4 *>(kd) = q0;
                *reinterpret_cast<uint4 *>(kd + 8) = q1;
            }
        }
        proxy_fence();
        tile_sync(g);
        // backward: W3^T (K = 16), then W2^T, W1^T (masked, rounded, kept), W0^T
        float dX[16];
        for (int layer = 3; layer >= 0 && ok; --layer) {
            if (layer == 3) ok = tc_layer(tmem, d4_addr, 256, wt_addr + 3 * 8192, 256, 64, 1, mbar, phase, u);
            else ok = tc_layer(tmem, a_addr, 1024, wt_addr + layer * 8192, 1024, 64, 4, mbar, phase, u);
            if (!ok) S.abort[g] = 1;
            tile_sync(g);
            if (S.abort[g]) { ok = false; break; }
            if (layer > 0) {
                const uint32_t mk = mask[layer - 1];     // the mask of the product's input
                uint16_t *kz = A.rb.dz + (int64_t)(layer - 1) * cap * 64 + i * 64;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float v[16];
                    tc_ld16(lane_addr + 16 * c, v);
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        float z[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) z[k] = (mk >> (16 * c + 8 * hh + k)) & 1u ? v[8 * hh + k] : 0.0f;
                        uint4 q;
                        q.x = pack2(z[0], z[1]);
                        q.y = pack2(z[2], z[3]);
                        q.z = pack2(z[4], z[5]);
                        q.w = pack2(z[6], z[7]);
                        const int col = 32 * hf + 16 * c + 8 * hh;
                        *reinterpret_cast<uint4 *>(arow + core_offset(r, col)) = q;
                        if (valid) *reinterpret_cast<uint4 *>(kz + col) = q;
                    }
                }
            } else {
                // input entries 16 hf .. 16 hf + 15: the gradient of this thread's levels
                float v[16];
                tc_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(16 * hf), v);
#pragma unroll
                for (int k = 0; k < 16; ++k) dX[k] = v[k];
            }
            tc_fence_before();
            proxy_fence();
            tile_sync(g);
        }
        if (!ok) break;
        if (valid) {
#pragma unroll 1
            for (int q = 0; q < 8; ++q) scatter_level(xn, 8 * hf + q, dX[2 * q], dX[2 * q + 1], A.dtable);
        }
    }
    loss = warp_sum_d(loss);
    if (lane == 0) S.red[warp] = loss;
    if (S.abort[g]) tc_drain(mbar, phase ^ 1u);      // the commit given up on is the pending phase
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < kTrainThreads / 32; ++w) sum += S.red[w];
        A.loss_part[blockIdx.x] = sum;
        int32_t any = 0;
        for (int k = 0; k < kTrainTiles; ++k) any |= S.abort[k];
        if (any) atomicOr(err, kErrTc);
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(S.tmem), "r"(kTrainCols)
                     : "memory");
}

int g_sms = 0;

}  // namespace

int train_grid(int device) {
    if (g_sms == 0) cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, device);
    return 2 * (g_sms > 0 ? g_sms : 1);
}

static cudaError_t set_smem(const void *fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_train(const TrainArgs &a, int grid, cudaStream_t s) {
    const size_t smem = smem_bytes(true);
    cudaError_t e = set_smem((const void *)train_kernel, smem);
    if (e != cudaSuccess) return e;
    train_kernel<<<grid, kMlpWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_train_tc(const TrainArgs &a, int32_t *err, cudaStream_t s, int *grid_out) {
    const size_t smem = sizeof(TcTrainSmem) + 1024;
    cudaError_t e = set_smem((const void *)train_tc_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t tiles = ((int64_t)a.batch + kTcRows - 1) / kTcRows;
    // as many CTAs as fit an SM's shared memory (two at two tiles per CTA)
    const int grid = (int)std::min<int64_t>((tiles + kTrainTiles - 1) / kTrainTiles,
                                            (int64_t)train_grid(dev) / 2 * kTrainCtasPerSm);
    *grid_out = grid;
    train_tc_kernel<<<grid, kTrainThreads, smem, s>>>(a, err);
    return cudaGetLastError();
}

cudaError_t launch_network(const NetworkArgs &a, cudaStream_t s) {
    const size_t smem = smem_bytes(true);
    cudaError_t e = set_smem((const void *)network_kernel, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = ((int64_t)a.rows + 15) / 16;
    const int grid = (int)std::min<int64_t>((tiles + kMlpWarps - 1) / kMlpWarps, 4096);
    network_kernel<<<grid, kMlpWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad(const RowBuffers &rb, int32_t rows, float *partial, float *dW, const double *loss_part,
                         int32_t n_loss_part, double *loss, cudaStream_t s) {
    const int chunks = (rows + kWgradChunk - 1) / kWgradChunk;
    wgrad_kernel<<<dim3(chunks, kWgradItems), 128, 0, s>>>(rb, rows, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wgrad_reduce_kernel<<<(kWeights + 255) / 256, 256, 0, s>>>(partial, chunks, dW, loss_part, n_loss_part, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, uint16_t *bf16_out, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    adam_kernel<<<grid, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, bf16_out);
    return cudaGetLastError();
}

cudaError_t launch_encode_points(const float *xn, int32_t n, const float *table, float *enc_out, cudaStream_t s) {
    const int64_t work = (int64_t)n * kLevels;
    encode_points_kernel<<<(int)((work + 255) / 256), 256, 0, s>>>(xn, n, table, enc_out);
    return cudaGetLastError();
}

cudaError_t launch_encode_texels(const TexelView &t, const float *table, uint16_t *enc, cudaStream_t s) {
    const int64_t work = t.n_pad * kLevels;
    encode_texels_kernel<<<(int)((work + 255) / 256), 256, 0, s>>>(t, table, enc);
    return cudaGetLastError();
}

static int design_grid(const DesignArgs &a) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t tiles = a.tex.n_pad / 16 * a.n_lights;
    return (int)std::min<int64_t>((tiles + kMlpWarps - 1) / kMlpWarps, (int64_t)train_grid(dev) * 4);
}

cudaError_t launch_design_forward(const DesignArgs &a, cudaStream_t s) {
    const size_t smem = smem_bytes(false);
    cudaError_t e = set_smem((const void *)design_forward_kernel, smem);
    if (e != cudaSuccess) return e;
    design_forward_kernel<<<design_grid(a), kMlpWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_design_reduce(const TexelView &t, const LightC *lights, int32_t n_lights, const float *K,
                                 const float *E_target, const float *alpha, float *E_out, float *up,
                                 double *loss_part, cudaStream_t s) {
    design_reduce_kernel<<<kReduceBlocks, 256, 0, s>>>(t, lights, n_lights, K, E_target, alpha, E_out, up, loss_part);
    return cudaGetLastError();
}

cudaError_t launch_design_forward_tc(const DesignArgs &a, int32_t *err, cudaStream_t s) {
    const size_t smem = sizeof(TcSmem) + 1024;
    cudaError_t e = set_smem((const void *)design_forward_tc_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t tiles = (a.tex.n_pad * (int64_t)a.n_lights + kTcRows - 1) / kTcRows;
    // two CTAs per SM (shared memory admits no third): 2 x 256 TMEM columns
    // never wait for an allocation
    const int grid = (int)std::min<int64_t>((tiles + kTcTiles - 1) / kTcTiles, (int64_t)train_grid(dev));
    design_forward_tc_kernel<<<grid, kTcThreads, smem, s>>>(a, err);
    return cudaGetLastError();
}

cudaError_t launch_design_backward_tc(const DesignArgs &a, int32_t *err, cudaStream_t s) {
    const size_t smem = sizeof(TcBwdSmem) + 1024;
    cudaError_t e = set_smem((const void *)design_backward_tc_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t tiles = (a.tex.n_pad * (int64_t)a.n_lights + kTcRows - 1) / kTcRows;
    // one CTA per SM (shared memory admits no second): kTcTiles x 64 TMEM
    // columns never wait for an allocation
    const int grid = (int)std::min<int64_t>((tiles + kTcTiles - 1) / kTcTiles, (int64_t)train_grid(dev) / 2);
    design_backward_tc_kernel<<<grid, kTcThreads, smem, s>>>(a, err);
    return cudaGetLastError();
}

cudaError_t launch_design_fused_tc(const DesignArgs &a, const FusedArgs &f, int32_t *err, cudaStream_t s,
                                   int *grid_out) {
    const size_t smem = sizeof(TcBwdSmem) + 1024;
    cudaError_t e = set_smem((const void *)design_fused_tc_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    // one CTA per SM (shared memory admits no second), as the design backward
    const int grid = (int)std::min<int64_t>((f.n_tiles + kTcTiles - 1) / kTcTiles, (int64_t)train_grid(dev) / 2);
    *grid_out = grid;
    design_fused_tc_kernel<<<grid, kTcThreads, smem, s>>>(a, f, err);
    return cudaGetLastError();
}

cudaError_t launch_design_backward(const DesignArgs &a, cudaStream_t s) {
    const size_t smem = smem_bytes(true);
    cudaError_t e = set_smem((const void *)design_backward_kernel, smem);
    if (e != cudaSuccess) return e;
    design_backward_kernel<<<design_grid(a), kMlpWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_design_final(const float *gpart, const LightC *lights, int32_t n_lights, int64_t tiles_per_light,
                                const double *loss_part, int32_t n_loss_part, double *out, cudaStream_t s) {
    design_final_kernel<<<n_lights + 1, 256, 0, s>>>(gpart, lights, n_lights, tiles_per_light, loss_part,
                                                     n_loss_part > 0 ? n_loss_part : kReduceBlocks, out);
    return cudaGetLastError();
}

}  // namespace sg
