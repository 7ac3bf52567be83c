// lt_internal.h -- device data layouts and launch interfaces shared by the
// library's own translation units (BVH builder, kernels, C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace lt {

constexpr int kWide = 8;                 // children per BVH node
constexpr int kMaxDepth = 16;            // levels of wide nodes (8-bit pending masks in two u64 words)
#ifndef LT_LEAF_MAX
#define LT_LEAF_MAX 3
#endif
constexpr int kLeafMax = LT_LEAF_MAX;    // triangles per leaf child (1..4)
static_assert(kLeafMax >= 1 && kLeafMax <= 4, "leaf encoding holds 1..4 triangles");
constexpr int32_t kEmptyChild = INT32_MIN;

// 8-wide BVH node, 240 bytes. Child boxes are stored axis-major (twelve
// 16-byte vectors), lo and hi of an axis 32 bytes apart, so a ray picks its
// near and far planes per axis by an address offset. child[k] >= 0 is an
// inner node index; a leaf is -1 - ((first << 2) | (count - 1)) over the
// leaf-ordered triangle array; kEmptyChild marks an unused slot, whose box is
// inverted (lo = +big, hi = -big) so that no ray ever hits it. Children sit
// in slots ordered by direction: bit a of the slot index is set when the
// child lies on the + side of the parent along axis a.
struct alignas(16) Node {
    float lox[kWide], hix[kWide], loy[kWide], hiy[kWide], loz[kWide], hiz[kWide];
    int32_t child[kWide];
    uint32_t inner_mask;     // slots holding inner nodes
    uint32_t pad[3];
};
static_assert(sizeof(Node) == 240, "node layout");
constexpr int kNodeVec = (int)(sizeof(Node) / 16);

// Compressed 8-wide node, 96 bytes, read by the kernels whose nodes come
// through L1 (quantised child boxes after Ylitie, Karras and Laine, HPG
// 2017). Per axis a: a float origin p[a] and a step 2^e_a; child k's planes
// are p[a] + q 2^e_a with the 8-bit q in q[a][k] (lo) and q[a][8 + k] (hi),
// rounded outward from the float node's (padded) planes by a further margin
// that covers the rounding of the kernel's decode. meta bytes 0-2 hold the
// biased exponents of 2^(e_a + 15) (so a plane decodes as one byte permute
// and one fma), byte 3 the inner mask. Empty slots have q lo = 255, q hi = 0,
// an inverted box. Slots and children as in Node.
struct alignas(16) CNode {
    float p[3];
    uint32_t meta;
    uint8_t q[3][16];
    int32_t child[kWide];
};
static_assert(sizeof(CNode) == 96, "compressed node layout");
constexpr int kCNodeVec = (int)(sizeof(CNode) / 16);

// Triangle in leaf order, 48 bytes (three 16-byte loads).
struct alignas(16) Tri {
    float v0[3];
    int32_t prim;     // index in the uploaded scene (ties in t go to the lower one)
    float v1[3];
    int32_t tile;
    float v2[3];
    float albedo;
};
static_assert(sizeof(Tri) == 48, "tri layout");
constexpr int kStagedTriBytes = 52;   // shared-memory stride of a staged triangle (13 words)

// What a hit needs besides the vertices: chart coordinates and texel range.
struct alignas(16) TriHit {
    float uv[6];
    int32_t res_u, res_v;
    int64_t texel_off;
    float n[3];              // unit geometric normal
    float pad[3];
};
static_assert(sizeof(TriHit) == 64, "hit layout");

// Per-light constants derived on the host (double, rounded to float).
struct alignas(16) LightDev {
    float pos[3];
    int32_t type;
    float ns[3];        // spot axis n(yaw, pitch)
    float flux_k;       // I_e * Omega / N_l: Phi_r = flux_k * a(theta)
    float e1[3];        // dn/dpitch
    float dflux_dp_k;   // p_int * Omega / N_l: dPhi_r/dp_int = dflux_dp_k * a(theta)
    float e2[3];        // dn/dyaw / cos(pitch)
    float co;           // cos(theta_out)
    float dn_dyaw[3];
    float ci;           // cos(theta_in)
    float dn_dpitch[3];
    float inv_d;        // 1 / (ci - co)
    float k_cos;        // emission cos = 1 - u1 k_cos: 2 (point), 1 - cos(theta_out) (spot), 1 (area)
    float sin_in;
    float sin_out;
    uint32_t design;    // design this light belongs to (Philox counter word 3, texel array)
    uint64_t first;     // global photon range [first, end)
    uint64_t end;
    uint64_t photon_base;   // first global photon of the light's design
    uint64_t texel_base;    // offset of the design's texel sums and weights (design slot x n_texels)
    float half_u, half_v;   // area light: half width along e1, half height along -e2
    float pad_area[2];
};
static_assert(sizeof(LightDev) == 160, "light layout");

// Values a captured step reads from device memory, so one instantiated graph
// serves every step (written with the lights from pinned host memory).
struct alignas(16) StepHeader {
    uint64_t seed_fwd;
    uint64_t seed_adj;
    double scale;       // fixed-point scale S of the texel sums
    double inv_scale;
    float flux_max;     // largest flux constant of the batch's lights (gradient scale anchor)
    float pad[3];
};

// What the adjoint trace keeps of one photon for the gradient kernel: the
// distance to its first hit along the emitted ray and 2 x first-hit
// triangle + 1 if the normal was flipped towards the light (-1: no hit),
// stored at the first hit, and its adjoint state dO/dPhi_r =
// sum_i w_{t_i} beta_i (Eq. 12), stored at the end of the path.
struct alignas(16) PhotonAdj {
    float t_first;
    int32_t n1code;
    float g;
    uint32_t pad;
};
static_assert(sizeof(PhotonAdj) == 16, "photon record layout");

// Device error word bits.
enum : int32_t { kErrSteps = 1, kErrRange = 2, kErrDepth = 4 };

struct TraceParams {
    const Node *nodes;          // float nodes (staged kernels)
    const CNode *cnodes;        // the same nodes compressed (kernels that read nodes through L1)
    const int32_t *parent;
    int32_t n_nodes;
    int32_t n_staged;           // nodes copied to shared memory by every block
    int32_t n_tris_staged;      // triangles copied there after the nodes (0: none; only with n_staged > 0)
    int32_t depth;              // levels of wide nodes (1..kMaxDepth)
    const Tri *tris;
    const TriHit *hits;
    const LightDev *lights;
    int32_t n_lights;
    int32_t max_hits;
    int32_t max_steps;          // node visits per ray before giving up (kErrSteps)
    uint64_t max_iters;         // step-loop iterations per thread before giving up (kErrSteps)
    uint64_t seed;
    const StepHeader *hdr;      // if set, seed and scale come from here (graph replay)
    uint64_t photon_begin, photon_end;
    int64_t n_texels;
    // forward
    unsigned long long *q;      // [designs][n_texels] fixed-point irradiance accumulator
    float scale;                // S
    uint64_t chunk;             // photons per thread (contiguous)
    // adjoint
    const float *w;             // [n_texels] dO/dPhi per deposit
    const uint32_t *wmax;       // bits of max_t |w_t| (gradient scale anchor, written by the weight-range kernel)
    float flux_max;             // largest flux constant of the lights (single-design passes; else hdr->flux_max)
    PhotonAdj *rec_adj;         // [photon_end - photon_begin] adjoint records (adjoint trace writes, gradient reads)
    ulonglong2 *slots;          // [threads][n_slots][8] gradient kernel's per-thread sums: 128-bit fixed point
    int32_t n_slots;            // lights a gradient thread's chunk can touch
    // debug record
    int32_t *rec_tri;
    int64_t *rec_texel;
    double *rec_grad;           // [count][8] per-photon gradient terms, may be null
    // counters
    unsigned long long *segments;
    unsigned long long *work;   // [2] node visits, triangle tests (counting kernel only)
    int32_t *err;
};

struct LossParams {
    const unsigned long long *q;    // [n_designs][n_texels]
    const float *E_target;          // shared by all designs
    const float *alpha;
    const float *area;
    double inv_scale;
    const StepHeader *hdr;          // if set, inv_scale comes from here
    int64_t n_texels;
    int32_t n_designs;
    float *E_out;                   // [n_designs][n_texels], may be null
    float *w_out;                   // [n_designs][n_texels]
    double *partial;                // [n_designs][kLossBlocks]
    double *loss_out;               // [n_designs] device
};

constexpr int kLossBlocks = 1024;
constexpr int kLossBlocksBatch = 128;   // blocks per design when several designs share a launch
constexpr int kLossThreads = 256;

// Kernel launchers (lt_kernels.cu).
cudaError_t launch_forward(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_forward_counted(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_adjoint(const TraceParams &p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_paths(const TraceParams &p, uint64_t count, cudaStream_t s);
cudaError_t launch_loss(const LossParams &p, cudaStream_t s);
cudaError_t launch_resolve(const unsigned long long *q, const float *area, double inv_scale, int64_t n,
                           float *E_out, cudaStream_t s);
// Gradient sums in two steps: n_lights x parts partial sums into `partial`
// ([n_lights][parts][8]), then one conversion per light.
cudaError_t launch_grad_finalize(const TraceParams &p, ulonglong2 *partial, int32_t parts, double *out,
                                 ulonglong2 *fixed_out, double *scale_out, cudaStream_t s);
// Partial sums per light: one per 1024 threads covering the light's photons
// (a light of max_nl photons in chunks of `chunk` spans up to
// ceil(max_nl / chunk) + 1 threads), at least 1, at most 256, so that a
// thread of the 256-thread partial blocks adds about four slots (one per
// 4096 threads, at most 64, left each thread a chain of 16 dependent slot
// loads: 24 us of a 0.22 ms Cornell box step).
inline int32_t grad_parts(uint64_t max_nl, uint64_t chunk) {
    const uint64_t threads = (max_nl + chunk - 1) / chunk + 1;
    const uint64_t parts = (threads + 1023) / 1024;
    return (int32_t)(parts < 1 ? 1 : (parts > 256 ? 256 : parts));
}
cudaError_t launch_weight_range(const float *w, int64_t n, uint32_t *wmax, cudaStream_t s);
// The gradient kernel: p.chunk photons per thread, p.n_slots slots each.
cudaError_t launch_grad_photons(const TraceParams &p, cudaStream_t s);
// Photons of one tracing pass at most: the kernels index a pass's photons
// and count a thread's segments and loop iterations in 32 bits.
constexpr uint64_t kMaxPassPhotons = 0xffffffffull;
constexpr uint64_t kGradPhotonsPerThread = 64;   // fewer for small passes (grad_params)
constexpr uint64_t kGradMinPhotonsPerThread = 3;
int trace_kernel_max_threads(bool staged);   // block bound of the staged / L1-node kernels
cudaError_t trace_occupancy(bool adjoint, bool staged, bool tris, int depth, int block, size_t smem,
                            int *blocks_per_sm);

// Wide-BVH builder (lt_bvh.cpp).
struct BvhBuild {
    std::vector<Node> nodes;        // breadth-first: parents before children
    std::vector<int32_t> parent;    // parent node of every node (-1 for the root)
    std::vector<int32_t> order;     // leaf-ordered triangle -> uploaded triangle index
    int depth = 0;
};
bool build_wide_bvh(const float *xyz, int32_t n_tri, BvhBuild *out, std::string *err);
// The compressed form of every node (false when a node is wider than about
// 2e6 along an axis, beyond the range of the kernels' decode).
bool compress_nodes(const Node *nodes, int32_t n_nodes, CNode *out);

}  // namespace lt
