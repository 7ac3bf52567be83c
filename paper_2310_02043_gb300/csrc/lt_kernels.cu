// lt_kernels.cu -- sm_103a kernels of view-independent adjoint light tracing
// (Lipp et al., arXiv 2310.02043): forward tracing into texels (Alg. 1,
// Eq. 7-8), the objective (Eq. 6), and the adjoint replay (Alg. 2,
// Eq. 11-15, S.11-S.12).
//
// Precision: FP32 throughout the path; fixed-point int64 texel sums; FP64
// gradient and loss reductions. The arithmetic that decides integers (which
// triangle is hit, which texel) uses explicitly rounded operations
// (__fmul_rn etc.) so the compiler cannot contract it into FMAs.
#include <cfloat>
#include <cstdint>

#include "../../include/lt.h"
#include "lt_internal.h"

namespace lt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Block shapes of the tracing kernels. With the whole BVH staged in shared
// memory, one block per SM holds it once and leaves the rest of the SM's
// shared storage to L1; 32 warps at 64 registers then beat 24 at 80.
// Kernels that read compressed nodes through L1 (BVHs too large to stage)
// run 32 warps at 64 registers as well: 7 % faster on the building than 24
// warps at 80 registers, which had won with float nodes. Both were chosen by
// measuring block shapes on GB300.
#ifndef LT_THREADS_STAGED
#define LT_THREADS_STAGED 1024
#endif
#ifndef LT_THREADS_L1
#define LT_THREADS_L1 1024
#endif
#ifndef LT_MIN_BLOCKS
#define LT_MIN_BLOCKS 1
#endif
constexpr int kThreadsStaged = LT_THREADS_STAGED;
constexpr int kThreadsL1 = LT_THREADS_L1;
constexpr int kTraceMinBlocks = LT_MIN_BLOCKS;   // resident blocks per SM the register budget targets
// Lanes by which a node step may trail leaf steps in a vote and still run
// (staged kernels; 4, 8 and 16 measured, 8 best).
constexpr int kNodeBias = 8;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The counter block of (photon, segment, design) under seed.
__device__ __forceinline__ uint4 counter_block(uint64_t seed, uint64_t photon, uint32_t segment, uint32_t design) {
    return philox(make_uint4((uint32_t)photon, (uint32_t)(photon >> 32), segment, design),
                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// A uniform in [0, 1) from the 24 high bits of one counter lane.
__device__ __forceinline__ float unit24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

// Four uniforms in [0, 1): lanes 0 and 1 give a direction, lanes 2 and 3
// the position on an area light.
__device__ __forceinline__ float4 uniforms(uint64_t seed, uint64_t photon, uint32_t segment, uint32_t design) {
    const uint4 r = counter_block(seed, photon, segment, design);
    return make_float4(unit24(r.x), unit24(r.y), unit24(r.z), unit24(r.w));
}

// 3-input min / max (PTX ISA 8.8, sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ---------------------------------------------------------------------------
// Rays
// ---------------------------------------------------------------------------
struct Ray {
    float ox, oy, oz;
    float dx, dy, dz;
    float ix, iy, iz;        // 1 / d, zero components replaced by +-1e-30
    int axes;                // watertight shear axes kx | ky << 2 | kz << 4
    int octant;              // bit a set when the ray runs towards -a
    float Sx, Sy, Sz;
};

__device__ __forceinline__ float sel3(float a, float b, float c, int k) { return k == 0 ? a : (k == 1 ? b : c); }

__device__ __forceinline__ void ray_init(Ray &r, float ox, float oy, float oz, float dx, float dy, float dz) {
    r.ox = ox; r.oy = oy; r.oz = oz;
    r.dx = dx; r.dy = dy; r.dz = dz;
    const float gx = fabsf(dx) < 1e-30f ? copysignf(1e-30f, dx) : dx;
    const float gy = fabsf(dy) < 1e-30f ? copysignf(1e-30f, dy) : dy;
    const float gz = fabsf(dz) < 1e-30f ? copysignf(1e-30f, dz) : dz;
    // 1/d for the slab tests only: an approximate reciprocal (1 ulp) scales a
    // ray's near and far distances along an axis alike, and the padding of
    // every child box covers the change of the plane distances, so no box the
    // ray touches is culled (the triangle test uses the exactly rounded shear
    // constants below)
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.ix) : "f"(gx));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.iy) : "f"(gy));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.iz) : "f"(gz));
    r.octant = (r.ix < 0.0f ? 1 : 0) | (r.iy < 0.0f ? 2 : 0) | (r.iz < 0.0f ? 4 : 0);
    int kz = 0;
    if (fabsf(dy) > fabsf(dx)) kz = 1;
    if (fabsf(dz) > fabsf(sel3(dx, dy, dz, kz))) kz = 2;
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    const float dkz = sel3(dx, dy, dz, kz);
    if (dkz < 0.0f) { const int t = kx; kx = ky; ky = t; }
    r.axes = kx | (ky << 2) | (kz << 4);
    r.Sx = __fdiv_rn(sel3(dx, dy, dz, kx), dkz);
    r.Sy = __fdiv_rn(sel3(dx, dy, dz, ky), dkz);
    r.Sz = __frcp_rn(dkz);
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013). Returns the
// unnormalised edge functions and determinant (det > 0) on a hit with t > 0.
struct TriTest {
    float t, U, V, W, det;
};

// The test proper, on the vertices relative to the ray origin with their
// coordinates already in the ray's shear order (kx, ky, kz).
__device__ __forceinline__ bool tri_sheared(const Ray &r, float Akx, float Aky, float Akz, float Bkx, float Bky,
                                            float Bkz, float Ckx, float Cky, float Ckz, TriTest &out) {
    const float Ax = __fsub_rn(Akx, __fmul_rn(r.Sx, Akz)), Ay = __fsub_rn(Aky, __fmul_rn(r.Sy, Akz));
    const float Bx = __fsub_rn(Bkx, __fmul_rn(r.Sx, Bkz)), By = __fsub_rn(Bky, __fmul_rn(r.Sy, Bkz));
    const float Cx = __fsub_rn(Ckx, __fmul_rn(r.Sx, Ckz)), Cy = __fsub_rn(Cky, __fmul_rn(r.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
        V = (float)__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
        W = (float)__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return false;
    const float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
    float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Az), __fmul_rn(V, Bz)), __fmul_rn(W, Cz));
    if (det < 0.0f) { det = -det; T = -T; U = -U; V = -V; W = -W; }
    if (!(T > 0.0f)) return false;
    out.t = __fdiv_rn(T, det);
    out.U = U; out.V = V; out.W = W; out.det = det;
    return true;
}

// ---------------------------------------------------------------------------
// Wide-BVH traversal without a stack. The pending children of every level
// are an 8-bit mask packed into registers (in the ray's visiting order, see
// order_mask); returning to a level follows the parent link and
// descends straight into the next pending child, without testing the
// parent's boxes again: a child that the closer hit found since would now
// cull is culled one level lower, by its own children's boxes, and CPU
// emulation of primary and bounce rays on the office and building BVHs
// shows that this visits 10-12 % fewer nodes than re-testing the parent.
// The pending masks of levels 0 .. depth - 2 (the deepest level's nodes
// have leaf children only) sit in one 32-bit word for trees of up to 5
// levels, in one 64-bit word for up to 9 and in two for up to kMaxDepth (the
// kTrail = 0, 1, 2 instantiations). Narrower words measured faster: 32 bits
// instead of 64 for the office's 5 levels -2 % forward time, one 64-bit word
// instead of two for the building's 9 levels -3 to -4 %.
// ---------------------------------------------------------------------------
// most levels of a tree each trail holds
__host__ __device__ constexpr int trail_levels(int kind) { return kind == 0 ? 5 : (kind == 1 ? 9 : kMaxDepth); }

__host__ __device__ constexpr int trail_kind(int depth) { return depth <= trail_levels(0) ? 0 : (depth <= trail_levels(1) ? 1 : 2); }

template <int kTrail>
struct Trail {
    uint64_t w0 = 0, w1 = 0;
    __device__ __forceinline__ uint32_t get(int lvl) const {
        const uint64_t w = lvl < 8 ? w0 : w1;
        return (uint32_t)(w >> ((lvl & 7) * 8)) & 0xffu;
    }
    __device__ __forceinline__ void set(int lvl, uint32_t m) {
        const int sh = (lvl & 7) * 8;
        const uint64_t clear = ~(0xffull << sh), put = (uint64_t)m << sh;
        if (lvl < 8) w0 = (w0 & clear) | put;
        else w1 = (w1 & clear) | put;
    }
};

template <>
struct Trail<1> {
    uint64_t w0 = 0;     // levels 0-7
    __device__ __forceinline__ uint32_t get(int lvl) const { return (uint32_t)(w0 >> (lvl * 8)) & 0xffu; }
    __device__ __forceinline__ void set(int lvl, uint32_t m) {
        const int sh = lvl * 8;
        w0 = (w0 & ~(0xffull << sh)) | ((uint64_t)m << sh);
    }
};

template <>
struct Trail<0> {
    uint32_t w0 = 0;     // levels 0-3
    __device__ __forceinline__ uint32_t get(int lvl) const { return (w0 >> (lvl * 8)) & 0xffu; }
    __device__ __forceinline__ void set(int lvl, uint32_t m) {
        const int sh = lvl * 8;
        w0 = (w0 & ~(0xffu << sh)) | (m << sh);
    }
};

struct Hit {
    int32_t tri;       // leaf-order index, -1 on a miss
    int32_t prim;      // uploaded index (tie-break)
    float t, b0, b1, b2;   // distance and barycentric weights of the three vertices
};

template <bool kHoldPrim>
__device__ __forceinline__ void take_hit(Hit &h, int32_t tri, int32_t prim, const TriTest &tt) {
    h.tri = tri; h.t = tt.t;
    if (kHoldPrim) h.prim = prim;
    h.b0 = __fdiv_rn(tt.U, tt.det);
    h.b1 = __fdiv_rn(tt.V, tt.det);
    h.b2 = __fdiv_rn(tt.W, tt.det);
}

struct Work {
    uint32_t nodes = 0, tris = 0;   // node visits and triangle tests
};

template <int kTrail>
struct Trav {
    int32_t node;       // node to test next, -1 when the traversal has no node left
    int32_t lvl;
    int32_t steps;
    int32_t leaf_node;  // node whose hit leaf children are pending
    uint32_t leaves;    // pending leaf children of leaf_node (slot order)
    int32_t leaf_node2; // a second node with pending leaves (speculative node steps only)
    uint32_t leaves2;
    Trail<kTrail> trail;
};

template <int kTrail>
__device__ __forceinline__ void trav_init(Trav<kTrail> &s, Hit &h) {
    s.node = 0; s.lvl = 0; s.steps = 0; s.leaf_node = 0; s.leaves = 0; s.leaf_node2 = 0; s.leaves2 = 0;
    s.trail = Trail<kTrail>();
    h.tri = -1; h.prim = INT32_MAX; h.t = FLT_MAX; h.b0 = h.b1 = h.b2 = 0.0f;
}

// Node loads: with kSmem every float node of the BVH sits in shared memory
// (the whole array was staged by the block, followed by the parent links);
// otherwise every node comes as a compressed node (CNode) from global memory
// through the read-only L1 path.
__device__ __forceinline__ const int32_t *staged_parent(const TraceParams &P, const float4 *smem) {
    return reinterpret_cast<const int32_t *>(smem + P.n_staged * kNodeVec);
}

// Triangles staged after the nodes and their parent links, when the launch
// stages them too: the 12 words of each Tri in leaf order, kTriWords (13)
// words apart. With an odd stride the same word of 32 different triangles
// falls into 32 different banks, so the leaf test's scalar loads from lanes
// at different triangles rarely conflict (a 12-word stride gives 8 bank
// classes; the odd stride measured 1.8 % faster on the office).
constexpr int kTriWords = kStagedTriBytes / 4;
__device__ __forceinline__ const float4 *staged_tris(const TraceParams &P, const float4 *smem) {
    return smem + P.n_staged * kNodeVec + (P.n_staged + 3) / 4;
}

// Word w (0..11) of staged triangle i.
__device__ __forceinline__ float staged_tri_word(const TraceParams &P, const float4 *smem, int32_t i, int w) {
    return reinterpret_cast<const float *>(staged_tris(P, smem))[kTriWords * i + w];
}

// Child word k of node n: staged float node, or compressed node through L1.
template <bool kSmem>
__device__ __forceinline__ int32_t child_word(const TraceParams &P, const float4 *smem, int32_t n, int k) {
    if (kSmem) return reinterpret_cast<const int32_t *>(smem + n * kNodeVec)[48 + k];
    return __ldg(reinterpret_cast<const int32_t *>(P.cnodes + n) + 16 + k);
}

// Ize, "Robust BVH ray traversal" (JCGT 2013): scale the exit distance by
// 1 + 2 gamma_3 so float rounding never rejects a box the ray touches.
constexpr float kFarScale = 1.0f + 2.0f * (3.0f * 0x1p-24f) / (1.0f - 3.0f * 0x1p-24f);

// Slab test of 4 children (slots 4h .. 4h+3) of a staged float node. The
// ray's near plane along an axis is lo when it runs towards +a and hi
// otherwise, so the entry and exit distances need no per-axis min/max: near
// and far planes are picked by address (lo and hi of an axis are two 16-byte
// vectors apart). A plane distance is one fma, plane * (1/d) + q with
// q = -o/d rounded once per node visit; the builder pads every child box by
// more than that rounding moves a plane, and the exit distance is scaled as
// in Ize's test, so no box the ray touches is rejected. The closest-hit
// bound is folded into the exit distance: tn <= min(tf, tbest).
__device__ __forceinline__ uint32_t test4(const float4 *smem, int32_t n, const Ray &r, float qx, float qy, float qz,
                                          float tbest, int half) {
    const int xn = (r.octant & 1) << 1, yn = 4 + (r.octant & 2), zn = 8 + ((r.octant & 4) >> 1);
    const float4 *v = smem + n * kNodeVec + half;
    const float4 nx = v[xn], fx = v[xn ^ 2], ny = v[yn], fy = v[yn ^ 2], nz = v[zn], fz = v[zn ^ 2];
    const float a_nx[4] = {nx.x, nx.y, nx.z, nx.w}, a_fx[4] = {fx.x, fx.y, fx.z, fx.w};
    const float a_ny[4] = {ny.x, ny.y, ny.z, ny.w}, a_fy[4] = {fy.x, fy.y, fy.z, fy.w};
    const float a_nz[4] = {nz.x, nz.y, nz.z, nz.w}, a_fz[4] = {fz.x, fz.y, fz.z, fz.w};
    uint32_t hit = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float tn = max3f(fmaf(a_nx[k], r.ix, qx), fmaf(a_ny[k], r.iy, qy), fmaxf(fmaf(a_nz[k], r.iz, qz), 0.0f));
        float tf = min3f(fmaf(a_fx[k], r.ix, qx), fmaf(a_fy[k], r.iy, qy), fmaf(a_fz[k], r.iz, qz)) * kFarScale;
        tf = fminf(tf, tbest);
        hit |= (tn <= tf ? 1u : 0u) << k;
    }
    return hit;
}

// Plane byte k (0..3) of a packed word of a compressed node, as the float
// 1 + q 2^-15 (exact: q lands in mantissa bits 8..15).
__device__ __forceinline__ float qplane(uint32_t word, int k) {
    return __uint_as_float(__byte_perm(word, 0x3F800000u, 0x7604u | ((uint32_t)k << 4)));
}

// Slab test of all 8 children of a compressed node read through L1 (four
// 16-byte loads). With E = 2^(e+15), plane p + q 2^e = p - E + (1 + q 2^-15) E,
// so its distance is fma(1 + q 2^-15, E/d, (p - E - o)/d): one byte permute
// and one fma per plane after three products per axis. The builder widens
// the quantised boxes by more than the decode's rounding moves a plane.
// Returns the hit mask (slot order) and the node's inner mask.
__device__ __forceinline__ uint32_t test_cnode(const TraceParams &P, int32_t n, const Ray &r, float tbest,
                                               uint32_t &inner) {
    const uint4 *cn = reinterpret_cast<const uint4 *>(P.cnodes + n);
    const uint4 hd = __ldg(cn);
    inner = hd.w >> 24;
    const uint4 vx = __ldg(cn + 1), vy = __ldg(cn + 2), vz = __ldg(cn + 3);
    const float Ex = __uint_as_float((hd.w & 0xffu) << 23), Ey = __uint_as_float(((hd.w >> 8) & 0xffu) << 23),
                Ez = __uint_as_float(((hd.w >> 16) & 0xffu) << 23);
    const float Sx = Ex * r.ix, Sy = Ey * r.iy, Sz = Ez * r.iz;
    const float Bx = ((__uint_as_float(hd.x) - Ex) - r.ox) * r.ix;
    const float By = ((__uint_as_float(hd.y) - Ey) - r.oy) * r.iy;
    const float Bz = ((__uint_as_float(hd.z) - Ez) - r.oz) * r.iz;
    const bool hx = r.octant & 1, hy = r.octant & 2, hz = r.octant & 4;   // near plane is hi
    uint32_t hit = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        // words: lo bytes of children 4h..4h+3, then their hi bytes 8 bytes on
        const uint32_t lx = h ? vx.y : vx.x, ux = h ? vx.w : vx.z;
        const uint32_t ly = h ? vy.y : vy.x, uy = h ? vy.w : vy.z;
        const uint32_t lz = h ? vz.y : vz.x, uz = h ? vz.w : vz.z;
        const uint32_t nx = hx ? ux : lx, fx = hx ? lx : ux;
        const uint32_t ny = hy ? uy : ly, fy = hy ? ly : uy;
        const uint32_t nz = hz ? uz : lz, fz = hz ? lz : uz;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float tn = max3f(fmaf(qplane(nx, k), Sx, Bx), fmaf(qplane(ny, k), Sy, By),
                                   fmaxf(fmaf(qplane(nz, k), Sz, Bz), 0.0f));
            float tf = min3f(fmaf(qplane(fx, k), Sx, Bx), fmaf(qplane(fy, k), Sy, By), fmaf(qplane(fz, k), Sz, Bz)) *
                       kFarScale;
            tf = fminf(tf, tbest);
            hit |= (tn <= tf ? 1u : 0u) << (4 * h + k);
        }
    }
    return hit;
}

// Child boxes of node n the ray enters before tbest (slot order), and the
// node's inner mask.
template <bool kSmem>
__device__ __forceinline__ uint32_t test_node(const TraceParams &P, const float4 *smem, int32_t n, const Ray &r,
                                              float tbest, uint32_t &inner) {
    if (!kSmem) return test_cnode(P, n, r, tbest, inner);
    inner = reinterpret_cast<const uint32_t *>(smem + n * kNodeVec)[56];
    const float qx = -r.ox * r.ix, qy = -r.oy * r.iy, qz = -r.oz * r.iz;
    return test4(smem, n, r, qx, qy, qz, tbest, 0) | (test4(smem, n, r, qx, qy, qz, tbest, 1) << 4);
}

// Mask in the ray's visiting order: slot s becomes bit s ^ octant, so the
// lowest set bit is the child on the side the ray comes from. The kernels
// look the permuted masks up in a 2 KB table in shared memory (8 octants x
// 256 masks; 2.8 % faster than the three conditional swaps per node visit),
// which every block fills first (fill_order_table, then a barrier).
__device__ __forceinline__ uint32_t order_mask_swaps(uint32_t m, int oct) {
    if (oct & 1) m = ((m & 0x55u) << 1) | ((m >> 1) & 0x55u);
    if (oct & 2) m = ((m & 0x33u) << 2) | ((m >> 2) & 0x33u);
    if (oct & 4) m = ((m & 0x0fu) << 4) | ((m >> 4) & 0x0fu);
    return m;
}

__shared__ uint8_t g_order_table[8 * 256];

__device__ __forceinline__ void fill_order_table() {
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x)
        g_order_table[i] = (uint8_t)order_mask_swaps((uint32_t)(i & 255), i >> 8);
}

__device__ __forceinline__ uint32_t order_mask(uint32_t m, int oct) { return g_order_table[(oct << 8) | m]; }

// Test the children of s.node; note hit leaves; descend to the first hit
// inner child in visiting order, or climb to the nearest level with pending
// children and descend into the first of them.
template <bool kCount, bool kSmem, int kTrail>
__device__ __forceinline__ void node_step(const TraceParams &P, const float4 *smem, const Ray &r, Trav<kTrail> &s, Hit &h,
                                          Work &work) {
    if (kCount) work.nodes += 1;
    if (++s.steps > P.max_steps) {
        atomicOr(P.err, kErrSteps);
        s.node = -1; s.leaves = 0; s.leaves2 = 0; h.tri = -1;
        return;
    }
    uint32_t inner;
    const uint32_t hit = test_node<kSmem>(P, smem, s.node, r, h.t, inner);
    const uint32_t leaves = hit & ~inner;
    if (leaves) {   // the second slot is taken only by a speculative step (first slot busy)
        if (!kSmem || s.leaves == 0) { s.leaf_node = s.node; s.leaves = leaves; }
        else { s.leaf_node2 = s.node; s.leaves2 = leaves; }
    }
    const uint32_t cand = order_mask(hit & inner, r.octant);
    if (cand) {
        if (s.lvl + 1 >= trail_levels(kTrail)) {   // deeper than the trail holds
            atomicOr(P.err, kErrDepth);
            s.node = -1; s.leaves = 0; s.leaves2 = 0; h.tri = -1;
            return;
        }
        const int j = __ffs(cand) - 1;
        s.trail.set(s.lvl, cand & ~(1u << j));
        s.node = child_word<kSmem>(P, smem, s.node, j ^ r.octant);
        ++s.lvl;
        return;
    }
    while (s.lvl > 0) {
        --s.lvl;
        s.node = kSmem ? staged_parent(P, smem)[s.node] : __ldg(P.parent + s.node);
        const uint32_t pend = s.trail.get(s.lvl);
        if (pend) {   // a level that was entered before, so lvl + 1 stays within the depth
            const int j = __ffs(pend) - 1;
            s.trail.set(s.lvl, pend & ~(1u << j));
            s.node = child_word<kSmem>(P, smem, s.node, j ^ r.octant);
            ++s.lvl;
            return;
        }
    }
    s.node = -1;
}

// Test the triangles of one pending leaf child. Ties in t go to the lower
// uploaded triangle index.
// kHoldPrim: keep the closest hit's uploaded index in a register for ties in
// t; otherwise read it back on a tie (rare), which frees a register (the
// forward kernels: building forward -2 %; the adjoint kernels keep it,
// where the freed register made the office 1 % slower).
template <bool kCount, bool kSmem, bool kTriSmem, int kTrail, bool kHoldPrim>
__device__ __forceinline__ void leaf_step(const TraceParams &P, const float4 *smem, const Ray &r, Trav<kTrail> &s, Hit &h,
                                          int32_t skip_tile, Work &work) {
    const int k = __ffs(s.leaves) - 1;
    s.leaves &= s.leaves - 1;
    const int32_t code = -1 - child_word<kSmem>(P, smem, s.leaf_node, k);
    if (kSmem && s.leaves == 0 && s.leaves2 != 0) { s.leaf_node = s.leaf_node2; s.leaves = s.leaves2; s.leaves2 = 0; }
    const int32_t first = code >> 2, count = (code & 3) + 1;
    // Each vertex coordinate is loaded by its own address in the ray's shear
    // order (kx, ky, kz), so the watertight test needs no selects to permute
    // the axes (office -6 % with the triangles staged, building -2 % through
    // L1, against three 16-byte loads per triangle and selects).
    if (kTriSmem) {
        const int kx = r.axes & 3, ky = (r.axes >> 2) & 3, kz = r.axes >> 4;
        const float okx = sel3(r.ox, r.oy, r.oz, kx), oky = sel3(r.ox, r.oy, r.oz, ky), okz = sel3(r.ox, r.oy, r.oz, kz);
        for (int32_t i = first; i < first + count; ++i) {
            const float *t = reinterpret_cast<const float *>(staged_tris(P, smem)) + kTriWords * i;
            if (__float_as_int(t[7]) == skip_tile) continue;
            if (kCount) work.tris += 1;
            const float *tx = t + kx, *ty = t + ky, *tz = t + kz;
            TriTest tt;
            if (!tri_sheared(r, __fsub_rn(tx[0], okx), __fsub_rn(ty[0], oky), __fsub_rn(tz[0], okz),
                             __fsub_rn(tx[4], okx), __fsub_rn(ty[4], oky), __fsub_rn(tz[4], okz),
                             __fsub_rn(tx[8], okx), __fsub_rn(ty[8], oky), __fsub_rn(tz[8], okz), tt))
                continue;
            const int32_t prim = __float_as_int(t[3]);
            if (tt.t < h.t || (tt.t == h.t && (kHoldPrim ? prim < h.prim
                                                      : (h.tri < 0 || prim < __float_as_int(staged_tri_word(P, smem, h.tri, 3))))))
                take_hit<kHoldPrim>(h, i, prim, tt);
        }
        return;
    }
    const int kx = r.axes & 3, ky = (r.axes >> 2) & 3, kz = r.axes >> 4;
    const float okx = sel3(r.ox, r.oy, r.oz, kx), oky = sel3(r.ox, r.oy, r.oz, ky), okz = sel3(r.ox, r.oy, r.oz, kz);
    for (int32_t i = first; i < first + count; ++i) {
        const float *t = reinterpret_cast<const float *>(P.tris + i);
        if (__float_as_int(__ldg(t + 7)) == skip_tile) continue;
        if (kCount) work.tris += 1;
        const float *tx = t + kx, *ty = t + ky, *tz = t + kz;
        TriTest tt;
        if (!tri_sheared(r, __fsub_rn(__ldg(tx), okx), __fsub_rn(__ldg(ty), oky), __fsub_rn(__ldg(tz), okz),
                         __fsub_rn(__ldg(tx + 4), okx), __fsub_rn(__ldg(ty + 4), oky), __fsub_rn(__ldg(tz + 4), okz),
                         __fsub_rn(__ldg(tx + 8), okx), __fsub_rn(__ldg(ty + 8), oky), __fsub_rn(__ldg(tz + 8), okz), tt))
            continue;
        const int32_t prim = __float_as_int(__ldg(t + 3));
        if (tt.t < h.t ||
            (tt.t == h.t && (kHoldPrim ? prim < h.prim
                                       : (h.tri < 0 || prim < __float_as_int(__ldg(reinterpret_cast<const float *>(P.tris + h.tri) + 3))))))
            take_hit<kHoldPrim>(h, i, prim, tt);
    }
}

// Closest hit excluding triangles of tile `skip_tile`, one ray at a time
// (path record); the same steps as the tracing kernels, so the same hits.
__device__ Hit closest_hit(const TraceParams &P, const float4 *smem, const Ray &r, int32_t skip_tile) {
    Trav<2> s;
    Hit h;
    Work work;
    trav_init(s, h);
    while (true) {
        if (s.leaves) leaf_step<false, false, false, 2, true>(P, smem, r, s, h, skip_tile, work);
        else if (s.node >= 0) node_step<false, false, 2>(P, smem, r, s, h, work);
        else return h;
    }
}

// Texel of a hit: barycentric chart coordinates in float, clamped,
// min(floor(u res), res - 1).
__device__ __forceinline__ int64_t texel_of(const TraceParams &P, const Hit &h) {
    const TriHit &th = P.hits[h.tri];
    float u = __fadd_rn(__fadd_rn(__fmul_rn(h.b0, th.uv[0]), __fmul_rn(h.b1, th.uv[2])), __fmul_rn(h.b2, th.uv[4]));
    float v = __fadd_rn(__fadd_rn(__fmul_rn(h.b0, th.uv[1]), __fmul_rn(h.b1, th.uv[3])), __fmul_rn(h.b2, th.uv[5]));
    u = u < 0.0f ? 0.0f : (u > 1.0f ? 1.0f : u);
    v = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
    int32_t iu = (int32_t)floorf(__fmul_rn(u, (float)th.res_u));
    int32_t iv = (int32_t)floorf(__fmul_rn(v, (float)th.res_v));
    iu = min(max(iu, 0), th.res_u - 1);
    iv = min(max(iv, 0), th.res_v - 1);
    return th.texel_off + (int64_t)iu + (int64_t)th.res_u * (int64_t)iv;
}

// Unit geometric normal of triangle `tri`, turned to face against w.
__device__ __forceinline__ float3 facing_normal(const TraceParams &P, int32_t tri, float wx, float wy, float wz) {
    const float *n = P.hits[tri].n;
    float nx = __ldg(n), ny = __ldg(n + 1), nz = __ldg(n + 2);
    if (nx * wx + ny * wy + nz * wz > 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
    return make_float3(nx, ny, nz);
}

__device__ __forceinline__ float albedo_of(const TraceParams &P, int32_t tri) {
    return __ldg(reinterpret_cast<const float *>(P.tris + tri) + 11);
}

__device__ __forceinline__ int32_t tile_of(const TraceParams &P, int32_t tri) {
    return __ldg(reinterpret_cast<const int32_t *>(P.tris + tri) + 7);
}

// Quadratic spot soft edge in cos(theta) (Eq. S.11).
__device__ __forceinline__ float falloff(const LightDev &L, float c) {
    if (L.type == LT_AREA) return c;            // Lambertian emitter: Phi_r proportional to cos
    if (c >= L.ci) return 1.0f;
    if (c <= L.co) return 0.0f;
    const float s = (c - L.co) * L.inv_d;
    return s * s;
}

__device__ __forceinline__ int32_t light_of(const TraceParams &P, uint64_t photon) {
    int32_t lo = 0, hi = P.n_lights - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (photon < P.lights[mid].end) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Direction with polar cosine c and sine s about n, azimuth 2 pi u2 measured
// from t1 towards t2. Emission and bounces share it; its operations are
// explicitly rounded so every kernel computes the same direction.
__device__ __forceinline__ float3 frame_dir(float c, float s, float u2, float3 t1, float3 t2, float3 n) {
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    const float a = __fmul_rn(s, cp), b = __fmul_rn(s, sp);
    return make_float3(__fmaf_rn(c, n.x, __fmaf_rn(b, t2.x, __fmul_rn(a, t1.x))),
                       __fmaf_rn(c, n.y, __fmaf_rn(b, t2.y, __fmul_rn(a, t1.y))),
                       __fmaf_rn(c, n.z, __fmaf_rn(b, t2.z, __fmul_rn(a, t1.z))));
}

// Emission frame and polar cosine of light L: uniform sphere (point: the
// world frame, cos = 1 - 2 u1) or uniform outer cone (spot: the axis frame,
// cos = 1 - u1 (1 - cos theta_out)); the host stores k_cos = 2 or
// 1 - cos theta_out and the world frame for point lights.
__device__ __forceinline__ void emit_frame(const LightDev &L, float u1, float &c, float &s, float3 &t1, float3 &t2,
                                           float3 &n) {
    c = 1.0f - u1 * L.k_cos;
    s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    t1 = make_float3(L.e1[0], L.e1[1], L.e1[2]);
    t2 = make_float3(L.e2[0], L.e2[1], L.e2[2]);
    n = make_float3(L.ns[0], L.ns[1], L.ns[2]);
}

// Cosine-weighted lobe about unit n: cos = sqrt(1 - u1), sin = sqrt(u1), with
// the branchless orthonormal basis of Duff et al. (JCGT 2017).
__device__ __forceinline__ void bounce_frame(float3 n, float u1, float &c, float &s, float3 &t1, float3 &t2) {
    const float sgn = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sgn + n.z);
    const float b = n.x * n.y * a;
    t1 = make_float3(1.0f + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
    t2 = make_float3(b, sgn + n.y * n.y * a, -n.y);
    c = sqrtf(1.0f - u1);
    s = sqrtf(u1);
}

// Coordinates of an area light's ray origin along e1 and b = -e2.
__device__ __forceinline__ float2 area_coords(const LightDev &L, float u3, float u4) {
    return make_float2((2.0f * u3 - 1.0f) * L.half_u, (2.0f * u4 - 1.0f) * L.half_v);
}

// Ray origin of light L: its position, or a uniform point of the rectangle.
__device__ __forceinline__ float3 emit_origin(const LightDev &L, float u3, float u4) {
    if (L.type != LT_AREA) return make_float3(L.pos[0], L.pos[1], L.pos[2]);
    const float2 q = area_coords(L, u3, u4);
    return make_float3(__fmaf_rn(-q.y, L.e2[0], __fmaf_rn(q.x, L.e1[0], L.pos[0])),
                       __fmaf_rn(-q.y, L.e2[1], __fmaf_rn(q.x, L.e1[1], L.pos[1])),
                       __fmaf_rn(-q.y, L.e2[2], __fmaf_rn(q.x, L.e1[2], L.pos[2])));
}

// Exitant ray of light L and its flux Phi_r = flux_k a(theta).
__device__ __forceinline__ float emit(const LightDev &L, float u1, float u2, float &wx, float &wy, float &wz,
                                      float &a) {
    float c, s;
    float3 t1, t2, n;
    emit_frame(L, u1, c, s, t1, t2, n);
    const float3 w = frame_dir(c, s, u2, t1, t2, n);
    wx = w.x; wy = w.y; wz = w.z;
    a = falloff(L, c);
    return L.flux_k * a;
}

__device__ __forceinline__ void cosine_dir(float3 n, float u1, float u2, float &wx, float &wy, float &wz) {
    float c, s;
    float3 t1, t2;
    bounce_frame(n, u1, c, s, t1, t2);
    const float3 w = frame_dir(c, s, u2, t1, t2, n);
    wx = w.x; wy = w.y; wz = w.z;
}

// Area light (supplement Eq. S.15-S.16): with the first hit x1 fixed and
// the origin x0 at fixed coordinates (su, sv) on the rectangle,
// dPhi_r/dq = I~ d(cos_1 / r^2)/dq + (2 P / N) d cos(theta)/dq, where x0
// translates with the centroid and turns with the axis (t = e1, b = -e2:
// dt/dyaw = -n_z e2, db/dyaw = t_z n - n_z t, dt/dpitch = -n).
__device__ __forceinline__ void area_dflux(const LightDev &L, float phi_r, float a_emit, float2 q, float x1x,
                                           float x1y, float x1z, float3 n1, float out[8]) {
    const float3 x0 = make_float3(L.pos[0] + q.x * L.e1[0] - q.y * L.e2[0], L.pos[1] + q.x * L.e1[1] - q.y * L.e2[1],
                                  L.pos[2] + q.x * L.e1[2] - q.y * L.e2[2]);
    const float dx = x0.x - x1x, dy = x0.y - x1y, dz = x0.z - x1z;
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float ux = dx * il, uy = dy * il, uz = dz * il;           // from x1 towards the origin
    const float c1 = n1.x * ux + n1.y * uy + n1.z * uz;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;                           // dPhi_r / dx0
    if (c1 > 0.0f) {
        const float k = phi_r * il, ic1 = 1.0f / c1;
        gx = k * (n1.x * ic1 - 3.0f * ux);
        gy = k * (n1.y * ic1 - 3.0f * uy);
        gz = k * (n1.z * ic1 - 3.0f * uz);
    }
    const float ct = -(L.ns[0] * ux + L.ns[1] * uy + L.ns[2] * uz);  // cos(theta) = n . w, w = -u
    const float kk = L.flux_k * il;                                   // 2 P / N / r
    gx -= kk * (L.ns[0] + ct * ux);
    gy -= kk * (L.ns[1] + ct * uy);
    gz -= kk * (L.ns[2] + ct * uz);
    out[0] = gx;
    out[1] = gy;
    out[2] = gz;
    const float nz = L.ns[2], tz = L.e1[2];
    float dyaw[3], dpitch[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dyaw[k] = -q.x * nz * L.e2[k] + q.y * (tz * L.ns[k] - nz * L.e1[k]);
        dpitch[k] = -q.x * L.ns[k];
    }
    const float w_dny = -(ux * L.dn_dyaw[0] + uy * L.dn_dyaw[1] + uz * L.dn_dyaw[2]);
    const float w_dnp = -(ux * L.dn_dpitch[0] + uy * L.dn_dpitch[1] + uz * L.dn_dpitch[2]);
    out[3] = gx * dyaw[0] + gy * dyaw[1] + gz * dyaw[2] + L.flux_k * w_dny;
    out[4] = gx * dpitch[0] + gy * dpitch[1] + gz * dpitch[2] + L.flux_k * w_dnp;
    out[5] = L.dflux_dp_k * a_emit;         // P = p^2 / 2
}

// dPhi_r/dp at the first hit x1 (normal n1 facing the light), the hit held
// fixed (Sec. 4.4.2). Order [x, y, z, yaw, pitch, p_int, theta_in, theta_out].
// q: the origin's coordinates on an area light.
__device__ __forceinline__ void dflux(const LightDev &L, float phi_r, float a_emit, float2 q, float x1x, float x1y,
                                      float x1z, float3 n1, float out[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] = 0.0f;
    if (L.type == LT_AREA) {
        area_dflux(L, phi_r, a_emit, q, x1x, x1y, x1z, n1, out);
        return;
    }
    const float dx = L.pos[0] - x1x, dy = L.pos[1] - x1y, dz = L.pos[2] - x1z;
    const float ell = sqrtf(dx * dx + dy * dy + dz * dz);
    const float il = 1.0f / ell;
    const float ux = dx * il, uy = dy * il, uz = dz * il;
    const float c1 = n1.x * ux + n1.y * uy + n1.z * uz;
    if (c1 > 0.0f) {
        // Eq. 14: virtual intensity Phi_r r^2 / cos times grad(cos / r^2)
        const float k = phi_r * il;
        const float ic1 = 1.0f / c1;
        out[0] = k * (n1.x * ic1 - 3.0f * ux);
        out[1] = k * (n1.y * ic1 - 3.0f * uy);
        out[2] = k * (n1.z * ic1 - 3.0f * uz);
    }
    out[5] = L.dflux_dp_k * a_emit;         // I_e = p^2 / 2
    if (L.type != LT_SPOT) return;
    const float wx = -ux, wy = -uy, wz = -uz;
    const float c = L.ns[0] * wx + L.ns[1] * wy + L.ns[2] * wz;
    if (!(c > L.co && c < L.ci)) return;
    const float scale = L.flux_k;            // I_e Omega / N_l
    const float s = (c - L.co) * L.inv_d;
    const float da_dc = 2.0f * s * L.inv_d;
    // Eq. S.12: d cos(theta)/dx = -(n - cos(theta) w) / r
    out[0] += scale * da_dc * (-(L.ns[0] - c * wx) * il);
    out[1] += scale * da_dc * (-(L.ns[1] - c * wy) * il);
    out[2] += scale * da_dc * (-(L.ns[2] - c * wz) * il);
    // Eq. 15 with n(yaw, pitch): d cos(theta)/dn = w
    out[3] = scale * da_dc * (wx * L.dn_dyaw[0] + wy * L.dn_dyaw[1] + wz * L.dn_dyaw[2]);
    out[4] = scale * da_dc * (wx * L.dn_dpitch[0] + wy * L.dn_dpitch[1] + wz * L.dn_dpitch[2]);
    const float id3 = L.inv_d * L.inv_d * L.inv_d;
    out[6] = scale * 2.0f * (c - L.co) * (c - L.co) * L.sin_in * id3;
    out[7] = scale * (-2.0f) * (c - L.co) * (c - L.ci) * L.sin_out * id3;
}

// Deposit (Eq. 8): one 64-bit fixed-point atomic. Lanes of a warp rarely hit
// the same 2-4.5 cm texel, so aggregating them first (__match_any_sync and
// shuffles) was measured slower (forward -1.5 % office, -3.9 % building);
// integer addition keeps the sums independent of the order either way.
__device__ __forceinline__ void deposit(unsigned long long *q, int64_t texel, unsigned long long val) {
    atomicAdd(q + texel, val);
}

// Seed and fixed-point scale of this launch: from the step header under
// graph replay, else from the launch parameters. Read where they are used
// rather than held across the loop, which keeps three registers free for
// the traversal state.
template <bool kAdjoint>
__device__ __forceinline__ uint64_t launch_seed(const TraceParams &P) {
    if (!P.hdr) return P.seed;
    return __ldg(kAdjoint ? &P.hdr->seed_adj : &P.hdr->seed_fwd);
}

__device__ __forceinline__ float launch_scale(const TraceParams &P) {
    return P.hdr ? (float)__ldg(&P.hdr->scale) : P.scale;
}

// ---------------------------------------------------------------------------
// Gradient sums in fixed point. Every photon's term g dPhi_r/dp (Eq. 11), a
// float, is scaled by a power of two G and rounded to a multiple of 2^-64
// (ties away from zero); the rounded terms are added as 128-bit
// two's-complement integers, so the sums do not depend on how photons are
// grouped into threads, launches or ranks. G = 2^-e with e the binary
// exponent of max_t |w_t| x (largest flux constant of the lights), the size
// of a typical term: a term 2^64 times smaller rounds away, and a term of
// 2^62 G^-1 or more, or one that is not finite, is an error.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float grad_scale(const TraceParams &P) {
    const float fm = P.hdr ? __ldg(&P.hdr->flux_max) : P.flux_max;
    const float t0 = __uint_as_float(__ldg(P.wmax)) * fm;
    int e = (int)((__float_as_uint(t0) >> 23) & 0xffu) - 127;   // floor(log2 t0) for a normal t0
    if (!(t0 > 0.0f)) e = 0;
    e = min(max(e, -120), 120);
    return __uint_as_float((uint32_t)(127 - e) << 23);           // 2^-e
}

// acc += round(v 2^64) as 128-bit two's complement (acc.x low, acc.y high
// word). False (nothing added) when |v| >= 2^62 or v is not finite.
__device__ __forceinline__ bool fix128_add(ulonglong2 &acc, float v) {
    const uint32_t b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) return true;                 // zero or below 2^-126: rounds to 0
    if (e >= 127 + 62) return false;         // |v| >= 2^62, inf or NaN
    const uint64_t m = (uint64_t)((b & 0x7fffffu) | 0x800000u);
    const int s = e - 86;                    // |v| 2^64 = m 2^(e - 86)
    uint64_t lo, hi;
    if (s < 0) {
        hi = 0;
        lo = s <= -25 ? 0 : (m + (1ull << (-s - 1))) >> (-s);
    } else if (s < 64) {
        lo = m << s;
        hi = s == 0 ? 0 : m >> (64 - s);
    } else {
        lo = 0;
        hi = m << (s - 64);
    }
    if (b >> 31) {
        lo = ~lo + 1;
        hi = ~hi + (lo == 0 ? 1 : 0);
    }
    const uint64_t nlo = acc.x + lo;
    acc.y += hi + (nlo < lo ? 1 : 0);
    acc.x = nlo;
    return true;
}

// 128-bit two's-complement integers as (low, high) words.
__device__ __forceinline__ void add128(ulonglong2 &a, ulonglong2 b) {
    const uint64_t lo = a.x + b.x;
    a.y += b.y + (lo < b.x ? 1 : 0);
    a.x = lo;
}

// The 128-bit integer as a double, rounded once (to nearest even).
__device__ __forceinline__ double int128_to_double(ulonglong2 v) {
    const bool neg = (int64_t)v.y < 0;
    uint64_t lo = v.x, hi = v.y;
    if (neg) {
        lo = ~lo + 1;
        hi = ~hi + (lo == 0 ? 1 : 0);
    }
    double d;
    if (hi == 0) {
        d = __ull2double_rn(lo);
    } else {
        const int n = __clzll((long long)hi);
        const uint64_t top = n == 0 ? hi : (hi << n) | (lo >> (64 - n));
        const uint64_t rest = lo << n;       // the bits below top; only whether any is set matters
        // top x 2^(64 - n), with the lost bits folded into top's last bit
        d = __ull2double_rn(top | (rest != 0 ? 1ull : 0ull)) * __longlong_as_double((long long)(1023 + 64 - n) << 52);
    }
    return neg ? -d : d;
}

__device__ __forceinline__ uint64_t thread_index() { return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; }

// One past the last photon of this thread's chunk.
__device__ __forceinline__ uint64_t thread_end(const TraceParams &P) {
    return P.photon_begin + min((thread_index() + 1) * P.chunk, P.photon_end - P.photon_begin);
}

// Every node and its parent link into shared memory, then (kTriSmem) every
// triangle; the caller syncs.
template <bool kTriSmem>
__device__ __forceinline__ void stage_nodes(const TraceParams &P, float4 *smem) {
    const int n = P.n_staged * kNodeVec;
    const float4 *src = reinterpret_cast<const float4 *>(P.nodes);
    for (int i = threadIdx.x; i < n; i += blockDim.x) smem[i] = __ldg(src + i);
    int32_t *parent = reinterpret_cast<int32_t *>(smem + n);
    for (int i = threadIdx.x; i < P.n_staged; i += blockDim.x) parent[i] = __ldg(P.parent + i);
    if (kTriSmem) {
        float *dst = reinterpret_cast<float *>(const_cast<float4 *>(staged_tris(P, smem)));
        const float *tsrc = reinterpret_cast<const float *>(P.tris);
        for (int i = threadIdx.x; i < 12 * P.n_tris_staged; i += blockDim.x)
            dst[(i / 12) * kTriWords + i % 12] = __ldg(tsrc + i);
    }
}

// ---------------------------------------------------------------------------
// Forward / adjoint tracing. Every thread owns a contiguous chunk of photons
// and advances its own path through a small state machine, one unit of work
// per loop iteration: test one BVH node, test the triangles of one leaf, or
// finish a segment (deposit / adjoint update, bounce, next photon). Each
// iteration the warp votes and runs the kind of step most of its lanes are
// waiting for, so lanes never idle until a neighbour's path ends.
// ---------------------------------------------------------------------------
template <bool kAdjoint, bool kCount, bool kSmem, bool kTriSmem, int kTrail>
__global__ void __launch_bounds__(kSmem ? kThreadsStaged : kThreadsL1, kTraceMinBlocks)
    trace_kernel(const TraceParams P) {
    static_assert(kSmem || !kTriSmem, "triangles are staged only with the nodes");
    extern __shared__ float4 smem[];
    fill_order_table();
    if (kSmem) stage_nodes<kTriSmem>(P, smem);
    __syncthreads();
    // The thread's photons are [begin + tid chunk, begin + (tid + 1) chunk)
    // clipped to the range; the end and the first photon's light are
    // recomputed where needed rather than held in registers.
    // photon indices relative to photon_begin: a pass covers fewer than 2^32
    // photons (kMaxPassPhotons), so 32 bits do, as for the thread's segment and
    // iteration counts (narrower state: 1-2 % faster, fewer spills)
    uint32_t pr = (uint32_t)min(thread_index() * P.chunk, P.photon_end - P.photon_begin);
    const uint32_t pr_end = (uint32_t)(thread_end(P) - P.photon_begin);

    int32_t l = 0, seg = 0, skip = -1;
    float phi = 0.0f, g = 0.0f, beta = 1.0f;
    Ray r;
    Trav<kTrail> s;
    Hit h;
    Work work;
    uint32_t segs = 0;
    bool active = pr < pr_end;

    // Emission of the first photon (Alg. 1: exitant ray carrying Phi_r).
    if (active) {
        l = light_of(P, P.photon_begin + pr);
        const LightDev &L = P.lights[l];
        const float4 u = uniforms(launch_seed<kAdjoint>(P), P.photon_begin + pr - L.photon_base, 0u, L.design);
        float wx, wy, wz, a_emit;
        phi = emit(L, u.x, u.y, wx, wy, wz, a_emit);
        const float3 o = emit_origin(L, u.z, u.w);
        ray_init(r, o.x, o.y, o.z, wx, wy, wz);
        seg = 1;
        trav_init(s, h);
    }

    uint32_t iters = 0;
    const uint32_t max_iters = (uint32_t)min(P.max_iters, (uint64_t)0xffffffffu);
    while (true) {
        // Every lane runs every iteration, so this count is warp-uniform; it
        // only trips if the step logic stops making progress.
        if (++iters > max_iters) {
            if ((threadIdx.x & 31) == 0) atomicOr(P.err, kErrSteps);
            break;
        }
        // With the BVH staged, a lane whose first leaf slot is busy still
        // takes node steps while its second slot is free (speculative
        // traversal, Aila and Laine, HPG 2009): node steps run with more
        // lanes, at the price of culling against an older closest hit.
        // Nodes read through L1 make that price higher than the gain, so
        // those kernels step a lane's leaves first.
        const bool can_leaf = active && s.leaves != 0;
        const bool can_node = active && (kSmem ? s.leaves2 == 0 : !can_leaf) && s.node >= 0;
        const bool fin = active && !can_leaf && s.node < 0;
        const unsigned bl = __ballot_sync(kFull, can_leaf);
        const unsigned bn = __ballot_sync(kFull, can_node);
        const unsigned bf = __ballot_sync(kFull, fin);
        if ((bl | bn | bf) == 0u) break;
        const int nl = __popc(bl), nn = __popc(bn), nf = __popc(bf);
        // The step kind with the most waiting lanes runs; in the staged
        // kernels node steps win ties with leaf steps up to kNodeBias lanes
        // (lanes with pending leaves can take either there). The chosen kind
        // always has a lane, so every iteration advances some lane.
        const int bias = kSmem ? kNodeBias : 0;
        int kind;
        if (nn > 0 && nn + bias >= nl && nn >= nf) kind = 0;
        else if (nl > 0 && nl >= nf) kind = 1;
        else if (nf > 0) kind = 2;
        else kind = nn > 0 ? 0 : 1;
        if (kind == 0) {
            if (can_node) node_step<kCount, kSmem, kTrail>(P, smem, r, s, h, work);
        } else if (kind == 1) {
            if (can_leaf) leaf_step<kCount, kSmem, kTriSmem, kTrail, kAdjoint>(P, smem, r, s, h, skip, work);
        } else if (fin) {
            // Finish the segment (one traced ray, hit or miss), then start the
            // next ray: a bounce from the hit or the next photon's emission.
            segs += 1;
            bool bounce = false;
            float3 x = make_float3(0.0f, 0.0f, 0.0f), nrm = make_float3(0.0f, 0.0f, 1.0f);
            if (h.tri >= 0) {
                const int64_t texel = texel_of(P, h);
                x = make_float3(fmaf(h.t, r.dx, r.ox), fmaf(h.t, r.dy, r.oy), fmaf(h.t, r.dz, r.oz));
                nrm = facing_normal(P, h.tri, r.dx, r.dy, r.dz);
                const uint64_t tb = P.lights[l].texel_base;
                if (!kAdjoint) {
                    deposit(P.q + tb, texel, (unsigned long long)__float2ll_rn(phi * launch_scale(P)));   // Eq. 8
                } else {
                    if (seg == 1) {   // the first hit: distance and 2 x triangle + flip bit
                        const int32_t n1code = 2 * h.tri + (nrm.x != __ldg(P.hits[h.tri].n) || nrm.y != __ldg(P.hits[h.tri].n + 1) ||
                                              nrm.z != __ldg(P.hits[h.tri].n + 2) ? 1 : 0);
                        *reinterpret_cast<float2 *>(&P.rec_adj[pr]) =
                            make_float2(h.t, __int_as_float(n1code));
                    }
                    g += __ldg(P.w + tb + texel) * beta;                                          // Eq. 12
                }
                if (seg < P.max_hits) {
                    const float rho = kTriSmem ? staged_tri_word(P, smem, h.tri, 11) : albedo_of(P, h.tri);
                    phi *= rho;                                                                 // Eq. 7
                    beta *= rho;
                    skip = kTriSmem ? __float_as_int(staged_tri_word(P, smem, h.tri, 7)) : tile_of(P, h.tri);
                    bounce = true;
                }
            }
            if (!bounce) {
                if (kAdjoint) {
                    // the photon's record for the gradient kernel (Eq. 11): its
                    // adjoint state dO/dPhi_r (Eq. 12) now; the first hit went
                    // in when it was found (two registers fewer along the path)
                    float2 *rp = reinterpret_cast<float2 *>(&P.rec_adj[pr]);
                    if (seg == 1 && h.tri < 0) rp[0] = make_float2(0.0f, __int_as_float(-1));   // no first hit
                    rp[1] = make_float2(g, 0.0f);
                }
                ++pr;
                if (pr >= pr_end) active = false;
            }
            if (active) {
                float c, sn;
                float3 t1, t2, axis, org;
                if (!bounce) while (P.photon_begin + pr >= P.lights[l].end) ++l;
                const LightDev &Ln = P.lights[l];
                const uint4 rb = counter_block(launch_seed<kAdjoint>(P), P.photon_begin + pr - Ln.photon_base, bounce ? (uint32_t)seg : 0u, Ln.design);
                const float2 u = make_float2(unit24(rb.x), unit24(rb.y));
                if (bounce) {
                    bounce_frame(nrm, u.x, c, sn, t1, t2);
                    axis = nrm;
                    org = x;
                    ++seg;
                } else {
                    emit_frame(Ln, u.x, c, sn, t1, t2, axis);
                    org = emit_origin(Ln, unit24(rb.z), unit24(rb.w));
                    phi = Ln.flux_k * falloff(Ln, c);
                    seg = 1;
                    skip = -1;
                    g = 0.0f;
                    beta = 1.0f;
                }
                const float3 w = frame_dir(c, sn, u.y, t1, t2, axis);
                ray_init(r, org.x, org.y, org.z, w.x, w.y, w.z);
                trav_init(s, h);
            }
        }
    }
    unsigned long long tot = segs;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(kFull, tot, off);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(P.segments, tot);
    if (kCount) {
        unsigned long long nodes = work.nodes, tris = work.tris;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            nodes += __shfl_xor_sync(kFull, nodes, off);
            tris += __shfl_xor_sync(kFull, tris, off);
        }
        if ((threadIdx.x & 31) == 0) { atomicAdd(P.work, nodes); atomicAdd(P.work + 1, tris); }
    }
}

// Eq. 11 per photon: thread t takes photons [begin + t K, begin + (t + 1) K)
// (K = P.chunk), recomputes each one's emitted ray from its Philox block (the
// same operations as at emission), its first hit x1 = o + t_first d and
// dPhi_r/dp there, and adds g dPhi_r/dp into 128-bit register sums for the
// photon's light; a light's run of photons ends in one store to the thread's
// slot for that light (slot = light - light of the thread's first photon).
// Slots of lights with no photon in the chunk are zero.
__global__ void __launch_bounds__(128) grad_photon_kernel(const TraceParams P) {
    const uint64_t n = P.photon_end - P.photon_begin;
    const uint64_t t = thread_index();
    uint64_t photon = P.photon_begin + min(t * P.chunk, n);
    const uint64_t p_end = P.photon_begin + min((t + 1) * P.chunk, n);
    ulonglong2 *slots = P.slots + t * (uint64_t)P.n_slots * 8;
    if (photon >= p_end) return;             // no photons: the slots are never read
    const float G = grad_scale(P);
    const uint64_t seed = launch_seed<true>(P);
    int32_t l = light_of(P, photon);
    ulonglong2 acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = make_ulonglong2(0, 0);
    bool in_range = true;
    for (int32_t s = 0; s < P.n_slots; ++s) {
        const LightDev &L = P.lights[l];
        const uint64_t stop = min(p_end, L.end);
        for (; photon < stop; ++photon) {
            const PhotonAdj rec = P.rec_adj[photon - P.photon_begin];
            if (rec.n1code < 0) continue;
            const uint4 r0 = counter_block(seed, photon - L.photon_base, 0u, L.design);
            float c0, s0;
            float3 e1, e2, ax;
            emit_frame(L, unit24(r0.x), c0, s0, e1, e2, ax);
            const float3 o0 = emit_origin(L, unit24(r0.z), unit24(r0.w));
            const float3 d0 = frame_dir(c0, s0, unit24(r0.y), e1, e2, ax);
            const float a_emit = falloff(L, c0);
            const float2 q = L.type == LT_AREA ? area_coords(L, unit24(r0.z), unit24(r0.w)) : make_float2(0.0f, 0.0f);
            const float *nn = P.hits[rec.n1code >> 1].n;
            const float sgn = (rec.n1code & 1) ? -1.0f : 1.0f;
            const float3 n1 = make_float3(sgn * __ldg(nn), sgn * __ldg(nn + 1), sgn * __ldg(nn + 2));
            float dp[8];
            dflux(L, L.flux_k * a_emit, a_emit, q, fmaf(rec.t_first, d0.x, o0.x), fmaf(rec.t_first, d0.y, o0.y),
                  fmaf(rec.t_first, d0.z, o0.z), n1, dp);
#pragma unroll
            for (int k = 0; k < 8; ++k) in_range &= fix128_add(acc[k], (rec.g * dp[k]) * G);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            slots[s * 8 + k] = acc[k];
            acc[k] = make_ulonglong2(0, 0);
        }
        if (photon < p_end) ++l;
    }
    if (!in_range) atomicOr(P.err, kErrRange);
}

// Path record for debugging: one thread per photon, the same per-segment
// arithmetic as the tracing kernels.
__global__ void __launch_bounds__(128) paths_kernel(const TraceParams P, uint64_t count) {
    fill_order_table();
    __syncthreads();
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint64_t photon = P.photon_begin + k;
    const int32_t l = light_of(P, photon);
    const LightDev &L = P.lights[l];
    float wx, wy, wz, a_emit;
    const uint64_t local = photon - L.photon_base;
    const float4 u0 = uniforms(P.seed, local, 0u, L.design);
    emit(L, u0.x, u0.y, wx, wy, wz, a_emit);
    const float3 o = emit_origin(L, u0.z, u0.w);
    const float2 q = L.type == LT_AREA ? area_coords(L, u0.z, u0.w) : make_float2(0.0f, 0.0f);
    int32_t skip = -1;
    int32_t *rt = P.rec_tri + k * P.max_hits;
    int64_t *rx = P.rec_texel + k * P.max_hits;
    for (int i = 0; i < P.max_hits; ++i) { rt[i] = -1; rx[i] = -1; }
    float g = 0.0f, beta = 1.0f;
    float x1x = 0.0f, x1y = 0.0f, x1z = 0.0f;
    float3 n1 = make_float3(0.0f, 0.0f, 0.0f);
    bool hit1 = false;
    Ray r;
    ray_init(r, o.x, o.y, o.z, wx, wy, wz);
    for (int i = 1; i <= P.max_hits; ++i) {
        const Hit h = closest_hit(P, nullptr, r, skip);
        if (h.tri < 0) break;
        const int64_t texel = texel_of(P, h);
        rt[i - 1] = h.prim;
        rx[i - 1] = texel;
        const float xx = fmaf(h.t, r.dx, r.ox), xy = fmaf(h.t, r.dy, r.oy), xz = fmaf(h.t, r.dz, r.oz);
        const float3 nrm = facing_normal(P, h.tri, r.dx, r.dy, r.dz);
        if (P.rec_grad) {
            if (i == 1) { x1x = xx; x1y = xy; x1z = xz; n1 = nrm; hit1 = true; }
            g += __ldg(P.w + L.texel_base + texel) * beta;
        }
        if (i == P.max_hits) break;
        const float4 u = uniforms(P.seed, local, (uint32_t)i, L.design);
        cosine_dir(nrm, u.x, u.y, wx, wy, wz);
        beta *= albedo_of(P, h.tri);
        skip = tile_of(P, h.tri);
        ray_init(r, xx, xy, xz, wx, wy, wz);
    }
    if (P.rec_grad) {
        float dp[8];
        for (int j = 0; j < 8; ++j) dp[j] = 0.0f;
        if (hit1) dflux(L, L.flux_k * a_emit, a_emit, q, x1x, x1y, x1z, n1, dp);
        for (int j = 0; j < 8; ++j) P.rec_grad[k * 8 + j] = (double)(g * dp[j]);
    }
}

// ---------------------------------------------------------------------------
// Objective (Eq. 6) and adjoint weights; fixed grid and fixed reduction order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    }
    __syncthreads();
    return t;
}

// blockIdx.y is the design; its texels are reduced by gridDim.x blocks.
__global__ void __launch_bounds__(kLossThreads) loss_kernel(const LossParams P) {
    __shared__ double sh[kLossThreads / 32];
    const int64_t base = (int64_t)blockIdx.y * P.n_texels;
    const double inv_scale = P.hdr ? P.hdr->inv_scale : P.inv_scale;
    double part = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P.n_texels;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double A = (double)P.area[t];
        const double E = (double)(long long)P.q[base + t] * inv_scale / A;
        const double r = E - (double)P.E_target[t];
        const double a = P.alpha ? (double)P.alpha[t] : 1.0;
        if (P.E_out) P.E_out[base + t] = (float)E;
        P.w_out[base + t] = (float)(a * r);
        part += 0.5 * A * a * r * r;
    }
    const double s = block_sum(part, sh);
    if (threadIdx.x == 0) P.partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// One block per design: the design's n block partials in order.
__global__ void __launch_bounds__(kLossThreads) loss_final_kernel(const double *partial, int n, double *out) {
    __shared__ double sh[kLossThreads / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[(int64_t)blockIdx.x * n + i];
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void resolve_kernel(const unsigned long long *q, const float *area, double inv_scale, int64_t n,
                               float *E) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        E[t] = (float)((double)(long long)q[t] * inv_scale / (double)area[t]);
}

// Sums of the per-thread 128-bit gradient slots, in two steps. Thread t's
// chunk of photons starts at begin + t * chunk and its slot s holds light
// (light of its first photon) + s. Step 1: block (l, p) of a grid of
// n_lights x P blocks sums every P-th group of 256 of the threads that cover
// light l into partial[l][p]. Step 2: one block per light, warp k summing
// component k of the P partials, writes the 128-bit sums (fixed_out), their
// value dO/dp = sum 2^-64 / G as
// doubles (out) and G (scale_out). Integer sums are exact, so neither the
// split nor the order of the additions changes a bit.
__global__ void __launch_bounds__(256) grad_partial_kernel(const TraceParams P, ulonglong2 *partial) {
    __shared__ ulonglong2 sh[256 / 32];
    const int32_t l = blockIdx.x;
    const uint32_t parts = gridDim.y, p = blockIdx.y;
    const uint64_t n = P.photon_end - P.photon_begin;
    const uint64_t lo = max(P.lights[l].first, P.photon_begin), hi = min(P.lights[l].end, P.photon_end);
    ulonglong2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = make_ulonglong2(0, 0);
    if (lo < hi && n > 0) {
        const uint64_t t0 = (lo - P.photon_begin) / P.chunk, t1 = (hi - 1 - P.photon_begin) / P.chunk;
        for (uint64_t t = t0 + (uint64_t)p * blockDim.x + threadIdx.x; t <= t1; t += (uint64_t)parts * blockDim.x) {
            const int32_t s = l - light_of(P, P.photon_begin + t * P.chunk);
            const ulonglong2 *src = P.slots + (t * (uint64_t)P.n_slots + (uint64_t)s) * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k) add128(v[k], src[k]);
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        ulonglong2 x = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ulonglong2 y;
            y.x = __shfl_xor_sync(kFull, x.x, off);
            y.y = __shfl_xor_sync(kFull, x.y, off);
            add128(x, y);
        }
        if (lane == 0) sh[w] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            ulonglong2 tot = make_ulonglong2(0, 0);
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) add128(tot, sh[i]);
            partial[((uint64_t)l * parts + p) * 8 + k] = tot;
        }
        __syncthreads();
    }
}

// One block of 8 warps per light, warp k summing component k.
__global__ void __launch_bounds__(256) grad_finalize_kernel(const TraceParams P, const ulonglong2 *partial,
                                                            int32_t parts, double *out, ulonglong2 *fixed_out,
                                                            double *scale_out) {
    const int32_t l = blockIdx.x;
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double unit = 0x1p-64 / (double)grad_scale(P);          // a power of two: exact
    ulonglong2 x = make_ulonglong2(0, 0);
    for (int32_t p = lane; p < parts; p += 32) add128(x, partial[((uint64_t)l * parts + p) * 8 + k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ulonglong2 y;
        y.x = __shfl_xor_sync(kFull, x.x, off);
        y.y = __shfl_xor_sync(kFull, x.y, off);
        add128(x, y);
    }
    if (lane == 0) {
        fixed_out[l * 8 + k] = x;
        out[l * 8 + k] = int128_to_double(x) * unit;
    }
    if (l == 0 && threadIdx.x == 0) scale_out[0] = (double)grad_scale(P);
}

// max_t |w_t| as float bits (non-negative floats order as unsigned integers)
// into *wmax, which the caller cleared.
__global__ void __launch_bounds__(256) weight_range_kernel(const float *w, int64_t n, uint32_t *wmax) {
    uint32_t m = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(w[t])));
    m = __reduce_max_sync(kFull, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(wmax, m);
}

template <class K>
cudaError_t allow_smem(K kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

using TraceFn = void (*)(TraceParams);

}  // namespace

int trace_kernel_max_threads(bool staged) { return staged ? kThreadsStaged : kThreadsL1; }

// The kernel instantiation for a launch: all nodes in shared memory when the
// launch stages the whole BVH, otherwise none, and the triangles too when
// the launch stages them; the narrowest trail of pending masks that holds
// the tree's levels.
template <bool kAdjoint, bool kCount, int kTrail>
TraceFn trace_fn_trail(bool staged, bool tris) {
    if (!staged) return trace_kernel<kAdjoint, kCount, false, false, kTrail>;
    return tris ? trace_kernel<kAdjoint, kCount, true, true, kTrail> : trace_kernel<kAdjoint, kCount, true, false, kTrail>;
}

template <bool kAdjoint, bool kCount>
TraceFn trace_fn(bool staged, bool tris, int depth) {
    switch (trail_kind(depth)) {
        case 0: return trace_fn_trail<kAdjoint, kCount, 0>(staged, tris);
        case 1: return trace_fn_trail<kAdjoint, kCount, 1>(staged, tris);
        default: return trace_fn_trail<kAdjoint, kCount, 2>(staged, tris);
    }
}

template <bool kAdjoint, bool kCount>
cudaError_t launch_trace(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    const TraceFn fn = trace_fn<kAdjoint, kCount>(p.n_staged > 0, p.n_tris_staged > 0, p.depth);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t trace_occupancy(bool adjoint, bool staged, bool tris, int depth, int block, size_t smem,
                            int *blocks_per_sm) {
    const TraceFn fn = adjoint ? trace_fn<true, false>(staged, tris, depth) : trace_fn<false, false>(staged, tris, depth);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t launch_forward(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    return launch_trace<false, false>(p, grid, block, smem, s);
}

cudaError_t launch_forward_counted(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    return launch_trace<false, true>(p, grid, block, smem, s);
}

cudaError_t launch_adjoint(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    return launch_trace<true, false>(p, grid, block, smem, s);
}

cudaError_t launch_paths(const TraceParams &p, uint64_t count, cudaStream_t s) {
    TraceParams q = p;
    q.n_staged = 0;
    q.n_tris_staged = 0;
    const unsigned blocks = (unsigned)((count + 127) / 128);
    paths_kernel<<<blocks, 128, 0, s>>>(q, count);
    return cudaGetLastError();
}

cudaError_t launch_loss(const LossParams &p, cudaStream_t s) {
    const int blocks = p.n_designs > 1 ? kLossBlocksBatch : kLossBlocks;
    loss_kernel<<<dim3(blocks, p.n_designs), kLossThreads, 0, s>>>(p);
    loss_final_kernel<<<p.n_designs, kLossThreads, 0, s>>>(p.partial, blocks, p.loss_out);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const unsigned long long *q, const float *area, double inv_scale, int64_t n, float *E,
                           cudaStream_t s) {
    resolve_kernel<<<1024, 256, 0, s>>>(q, area, inv_scale, n, E);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const TraceParams &p, ulonglong2 *partial, int32_t parts, double *out,
                                 ulonglong2 *fixed_out, double *scale_out, cudaStream_t s) {
    grad_partial_kernel<<<dim3(p.n_lights, parts), 256, 0, s>>>(p, partial);
    grad_finalize_kernel<<<p.n_lights, 256, 0, s>>>(p, partial, parts, out, fixed_out, scale_out);
    return cudaGetLastError();
}

cudaError_t launch_grad_photons(const TraceParams &p, cudaStream_t s) {
    const uint64_t n = p.photon_end - p.photon_begin;
    const uint64_t threads = (n + p.chunk - 1) / p.chunk;
    if (threads == 0) return cudaSuccess;
    grad_photon_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_weight_range(const float *w, int64_t n, uint32_t *wmax, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(wmax, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    weight_range_kernel<<<1024, 256, 0, s>>>(w, n, wmax);
    return cudaGetLastError();
}

}  // namespace lt
