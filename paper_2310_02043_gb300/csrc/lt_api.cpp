// lt_api.cpp -- the C ABI declared in include/lt.h: context, device buffers,
// scene/BVH upload, light constants, launches and error reporting.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lt.h"
#include "lt_internal.h"

namespace {

using namespace lt;

constexpr double kPi = 3.14159265358979323846;

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    // scene
    Node *d_nodes = nullptr;
    CNode *d_cnodes = nullptr;             // the same nodes compressed (kernels reading nodes through L1)
    int32_t *d_parent = nullptr;
    Tri *d_tris = nullptr;
    TriHit *d_hits = nullptr;
    float *d_area = nullptr;
    int32_t n_nodes = 0, n_tri = 0, depth = 0;
    int64_t n_texels = 0;
    std::vector<float> tile_area_f;    // texel area per tile (float)
    // objective
    float *d_target = nullptr, *d_alpha = nullptr;
    bool has_target = false, has_alpha = false;
    // lights
    std::vector<lt_light> lights;
    uint32_t design_word = 0;          // Philox counter word 3 of the single-design passes
    LightDev *d_lights = nullptr;       // [LT_MAX_LIGHTS]
    LightDev *h_lights = nullptr;       // pinned staging of the same size
    cudaEvent_t lights_copied = nullptr;
    uint64_t lights_for_n = 0;         // photon budget the device light table was built for
    bool lights_dirty = true;
    double power_bound = 0.0;          // sum_l I_l Omega_l
    // pass state
    unsigned long long *d_q = nullptr;
    float *d_E = nullptr, *d_w = nullptr;
    double scale = 1.0;
    bool fwd_done = false, has_w = false;
    double *d_loss = nullptr, *d_partial = nullptr, *d_grad = nullptr;
    ulonglong2 *d_slots = nullptr;         // gradient kernel's per-thread sums (128-bit fixed point)
    size_t slots_bytes = 0;
    PhotonAdj *d_rec = nullptr;            // per-photon adjoint records of the last adjoint pass
    size_t rec_bytes = 0;
    ulonglong2 *d_gpart = nullptr;         // [lights][parts][8] partial gradient sums
    size_t gpart_bytes = 0;
    ulonglong2 *d_gfix = nullptr;          // [LT_MAX_LIGHTS][8] exact gradient sums of the last adjoint pass
    double *d_gscale = nullptr;            // their scale G
    uint32_t *d_wmax = nullptr;            // max |w_t| (float bits) of the last adjoint pass
    float flux_max = 0.0f;                 // largest flux constant of the uploaded lights
    int32_t adj_lights = 0;                // lights of the last adjoint pass (0: none yet)
    unsigned long long *d_seg = nullptr;   // [2]: forward, adjoint
    int32_t *d_err = nullptr;
    double *h_pinned = nullptr;            // small pinned staging area
    // launch
    int threads = 0, blocks_per_sm = 0, smem_node_bytes = 72 * 1024;   // threads 0: the kernel's bound
    int smem_tri_bytes = 200 * 1024;       // triangles staged when nodes + parent links + triangles fit this
    int32_t max_steps = 0;                 // node visits per ray before giving up; 0: 16 x nodes + 64
    lt_stats stats{};
    // host copy of the uploaded charts (texel centres)
    std::vector<float> h_xyz, h_uv;
    std::vector<int32_t> h_tile, h_res;
    std::vector<int64_t> h_off;
    bool seg_single = true;                // segment counters in d_seg belong to the last pass
    // batched designs (lt_batch_*)
    struct Batch {
        int32_t n_designs = 0, n_lights = 0, max_hits = 0;
        uint64_t photons = 0;                 // per design
        std::vector<int32_t> counts;          // lights per design
        std::vector<lt_light> lights;         // concatenated
        bool has_lights = false;
        cudaStream_t stream = nullptr;        // private, capturable
        unsigned char *d_in = nullptr;        // StepHeader + LightDev[n_lights]
        unsigned char *h_in = nullptr;        // pinned copy the step uploads
        double *h_out = nullptr;              // pinned: loss[n_designs], grad[n_lights][8]
        unsigned long long *d_q = nullptr;
        float *d_E = nullptr, *d_w = nullptr;
        double *d_partial = nullptr, *d_loss = nullptr, *d_grad = nullptr;
        ulonglong2 *d_slots = nullptr;
        PhotonAdj *d_rec = nullptr;
        size_t rec_bytes = 0;
        ulonglong2 *d_gfix = nullptr;         // [n_lights][8] exact gradient sums
        ulonglong2 *d_gpart = nullptr;        // [n_lights][parts][8] partial gradient sums
        size_t gpart_bytes = 0;
        double *d_gscale = nullptr;
        uint32_t *d_wmax = nullptr;
        size_t in_bytes = 0, slots_bytes = 0;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        uint64_t segments = 0;
    } batch;
};

// An NVTX range around an entry point, so profiler timelines show the ABI
// calls with the kernels they launch (no cost without an attached tool).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

int fail(Ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

// No C++ exception crosses the C ABI: every entry point runs its body between
// LT_TRY and LT_CATCH, which turn an exception into a status and, when there
// is a context, its message. Called only from inside a catch handler.
int exception_status(Ctx *c) noexcept {
    int code = LT_ERR_STATE;
    const char *msg = "unexpected C++ exception";
    try {
        throw;
    } catch (const std::bad_alloc &) {
        code = LT_ERR_OOM;
        msg = "host memory exhausted";
    } catch (const std::length_error &) {
        code = LT_ERR_ARG;
        msg = "a size exceeds what a host container can hold";
    } catch (...) {
    }
    if (c) {
        try {
            c->err = msg;
        } catch (...) {
        }
    }
    return code;
}

// Host-side fault injection for testing callers' error paths: with the
// environment variable LT_FAULT_HOST_ALLOC set and non-empty, the host
// allocations of a BVH build fail as if memory ran out.
void maybe_inject_host_oom() {
    const char *v = std::getenv("LT_FAULT_HOST_ALLOC");
    if (v && v[0]) throw std::bad_alloc();
}

#define LT_TRY try {
#define LT_CATCH(ctx)                                      \
    }                                                      \
    catch (...) {                                          \
        return exception_status(static_cast<Ctx *>(ctx));  \
    }

int cuda_fail(Ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define LT_CUDA(c, expr)                                   \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
    } while (0)

template <class T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <class T>
cudaError_t dalloc(T *&p, size_t n) {
    dfree(p);
    if (n == 0) n = 1;
    return cudaMalloc(reinterpret_cast<void **>(&p), n * sizeof(T));
}

// Status of a non-zero device error word.
int device_error(Ctx *c, int32_t e) {
    if (e & kErrSteps) return fail(c, LT_ERR_TIMEOUT, "a ray exceeded its traversal step limit");
    if (e & kErrRange)
        return fail(c, LT_ERR_OVERFLOW, "a photon's gradient term is not finite or beyond the fixed-point range");
    return fail(c, LT_ERR_DEVICE, "kernel error word " + std::to_string(e));
}

// Reads the device error word (synchronises the stream) and clears it.
int check_device(Ctx *c) {
    int32_t e = 0;
    LT_CUDA(c, cudaMemcpyAsync(&e, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    LT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (e) {
        LT_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream));
        return device_error(c, e);
    }
    return LT_OK;
}

int copy_in(Ctx *c, void *dst, const void *src, size_t bytes, int is_device) {
    LT_CUDA(c, cudaMemcpyAsync(dst, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c->stream));
    return LT_OK;
}

int copy_out(Ctx *c, void *dst, const void *src, size_t bytes, int is_device) {
    LT_CUDA(c, cudaMemcpyAsync(dst, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               c->stream));
    if (!is_device) LT_CUDA(c, cudaStreamSynchronize(c->stream));
    return LT_OK;
}

// Per-light constants of one design whose photon budget n is split evenly
// over its L lights (Sec. 4.4 and the supplement): I_e = p^2 / 2,
// Phi_r = I_e Omega a / N_l with Omega = 4 pi (point), 2 pi (1 - cos
// theta_out) (spot, a the soft edge) or 2 (area: P = p^2 / 2, a = cos theta,
// Phi_r = 2 P cos / N_l). The design's photons are global indices
// [photon_base, photon_base + n); its texel arrays start at texel_base.
// Returns the design's power bound sum_l I_l Omega_l.
double derive_lights(const lt_light *in, int32_t L, uint64_t n_photons, uint64_t photon_base, uint64_t texel_base,
                     uint32_t design, LightDev *out) {
    const uint64_t base = n_photons / (uint64_t)L, rem = n_photons % (uint64_t)L;
    uint64_t first = photon_base;
    double bound = 0.0;
    for (int32_t l = 0; l < L; ++l) {
        const lt_light &s = in[l];
        LightDev &d = out[l];
        std::memset(&d, 0, sizeof(d));
        const uint64_t nl = base + ((uint64_t)l < rem ? 1u : 0u);
        const double I = 0.5 * (double)s.p_int * (double)s.p_int;
        const double cy = std::cos((double)s.yaw), sy = std::sin((double)s.yaw);
        const double cp = std::cos((double)s.pitch), sp = std::sin((double)s.pitch);
        double omega = 4.0 * kPi;
        d.type = s.type;
        for (int k = 0; k < 3; ++k) d.pos[k] = s.pos[k];
        d.ns[0] = (float)(cp * cy); d.ns[1] = (float)(cp * sy); d.ns[2] = (float)sp;
        d.e1[0] = (float)(-sp * cy); d.e1[1] = (float)(-sp * sy); d.e1[2] = (float)cp;
        d.e2[0] = (float)(-sy); d.e2[1] = (float)cy; d.e2[2] = 0.0f;
        d.dn_dyaw[0] = (float)(-cp * sy); d.dn_dyaw[1] = (float)(cp * cy); d.dn_dyaw[2] = 0.0f;
        d.dn_dpitch[0] = (float)(-sp * cy); d.dn_dpitch[1] = (float)(-sp * sy); d.dn_dpitch[2] = (float)cp;
        if (s.type == LT_SPOT) {
            const double co = std::cos((double)s.theta_out), ci = std::cos((double)s.theta_in);
            omega = 2.0 * kPi * (1.0 - co);
            d.co = (float)co;
            d.ci = (float)ci;
            d.inv_d = (float)(1.0 / (ci - co));
            d.k_cos = (float)(1.0 - co);
            d.sin_in = (float)std::sin((double)s.theta_in);
            d.sin_out = (float)std::sin((double)s.theta_out);
        } else if (s.type == LT_AREA) {
            // the hemisphere about n; the falloff is the emission cosine
            omega = 2.0;
            d.k_cos = 1.0f;
            d.ci = 2.0f;
            d.co = 0.0f;
            d.inv_d = 1.0f;
            d.half_u = 0.5f * s.theta_in;
            d.half_v = 0.5f * s.theta_out;
        } else {
            // point light: the whole sphere about the world z axis, no falloff
            d.e1[0] = 1.0f; d.e1[1] = 0.0f; d.e1[2] = 0.0f;
            d.e2[0] = 0.0f; d.e2[1] = 1.0f; d.e2[2] = 0.0f;
            d.ns[0] = 0.0f; d.ns[1] = 0.0f; d.ns[2] = 1.0f;
            d.k_cos = 2.0f;
            d.ci = -2.0f;
            d.co = -3.0f;
            d.inv_d = 1.0f;
        }
        d.flux_k = nl ? (float)(I * omega / (double)nl) : 0.0f;
        d.dflux_dp_k = nl ? (float)((double)s.p_int * omega / (double)nl) : 0.0f;
        d.first = first;
        d.end = first + nl;
        d.design = design;
        d.photon_base = photon_base;
        d.texel_base = texel_base;
        first += nl;
        bound += I * omega;
    }
    return bound;
}

// Grows a device buffer to at least `bytes` (waits for `s` before freeing the
// old one, whose contents are not kept). Sets *grown when it reallocated.
template <class T>
int grow(Ctx *c, T *&buf, size_t &cap, size_t bytes, cudaStream_t s, bool *grown = nullptr) {
    if (bytes <= cap) return LT_OK;
    LT_CUDA(c, cudaStreamSynchronize(s));
    dfree(buf);
    LT_CUDA(c, cudaMalloc(reinterpret_cast<void **>(&buf), bytes));
    cap = bytes;
    if (grown) *grown = true;
    return LT_OK;
}

// Launch parameters of the gradient kernel (Eq. 11) after an adjoint trace
// over the photons of `p`: kGradPhotonsPerThread photons per thread, or fewer
// for a pass too small to give every SM 1024 threads that way, but at least
// kGradMinPhotonsPerThread: every thread writes 128 bytes of 128-bit sums per
// slot, which at one photon per thread outweigh the 16-byte photon records
// (Cornell box, 2^18 photons, adjoint with 1, 3, 6 and 13 photons per
// thread: 0.129, 0.123, 0.125 and 0.135 ms); and a slot per light that a
// thread's chunk can touch (chunk / fewest photons of a light + 2, at most
// all lights).
TraceParams grad_params(const TraceParams &p, uint64_t min_photons_per_light, ulonglong2 *slots, int sm_count) {
    TraceParams g = p;
    const uint64_t n = p.photon_end - p.photon_begin, full = (uint64_t)std::max(sm_count, 1) * 1024;
    g.chunk = n >= kGradPhotonsPerThread * full ? kGradPhotonsPerThread
                                                : std::max<uint64_t>(kGradMinPhotonsPerThread, n / full);
    g.n_slots = min_photons_per_light == 0
                    ? p.n_lights
                    : (int32_t)std::min<uint64_t>((uint64_t)p.n_lights, g.chunk / min_photons_per_light + 2);
    g.slots = slots;
    return g;
}

size_t grad_slot_bytes(const TraceParams &g) {
    const uint64_t n = g.photon_end - g.photon_begin;
    return (size_t)((n + g.chunk - 1) / g.chunk) * (size_t)g.n_slots * 8 * sizeof(ulonglong2);
}

// Largest flux constant of n derived lights: with the largest adjoint weight
// it sets the size of a typical gradient term and so the gradient scale.
float max_flux(const LightDev *lights, int32_t n) {
    float m = 0.0f;
    for (int32_t l = 0; l < n; ++l) m = std::max(m, std::fabs(lights[l].flux_k));
    return m;
}

int upload_lights(Ctx *c, uint64_t n_photons) {
    if (!c->lights_dirty && c->lights_for_n == n_photons) return LT_OK;
    const int32_t L = (int32_t)c->lights.size();
    // the previous copy out of the staging buffer must be done before reuse
    LT_CUDA(c, cudaEventSynchronize(c->lights_copied));
    LightDev *h = c->h_lights;
    const double bound = derive_lights(c->lights.data(), L, n_photons, 0, 0, c->design_word, h);
    c->flux_max = max_flux(h, L);
    LT_CUDA(c, cudaMemcpyAsync(c->d_lights, h, sizeof(LightDev) * (size_t)L, cudaMemcpyHostToDevice, c->stream));
    LT_CUDA(c, cudaEventRecord(c->lights_copied, c->stream));
    c->lights_for_n = n_photons;
    c->lights_dirty = false;
    c->power_bound = bound;
    return LT_OK;
}

// Launch shape of a tracing kernel. The whole BVH is staged in shared memory
// when it fits the budget, otherwise no node is (nodes then come through L1);
// with the nodes staged, the triangles follow them when nodes and triangles
// together fit the triangle budget and the extra shared memory costs no
// resident block (the requested blocks per SM, else as many as fit without
// the triangles). Sets p->n_staged and p->n_tris_staged. The block is the
// requested size, else the bound of the kernel chosen.
int launch_shape(Ctx *c, bool adjoint, int *grid, int *threads, size_t *smem, TraceParams *p) {
    const bool staged = (int64_t)c->n_nodes * (int64_t)sizeof(Node) <= (int64_t)c->smem_node_bytes;
    p->n_staged = staged ? c->n_nodes : 0;
    // staged nodes, then their parent links (int32, rounded up to 16 bytes)
    *smem = (size_t)p->n_staged * sizeof(Node) + ((size_t)p->n_staged + 3) / 4 * 16;
    const int bound = trace_kernel_max_threads(staged);
    *threads = c->threads > 0 ? c->threads : bound;
    if (*threads > bound)
        return fail(c, LT_ERR_ARG, "threads_per_block " + std::to_string(*threads) + " exceeds the bound " +
                                       std::to_string(bound) + " of the kernel for this BVH");
    const size_t tri_bytes = ((size_t)c->n_tri * kStagedTriBytes + 15) / 16 * 16;
    bool tris = staged && *smem + tri_bytes <= (size_t)c->smem_tri_bytes;
    if (tris) {
        int with = 0, without = 0;
        cudaError_t e = trace_occupancy(adjoint, true, true, c->depth, *threads, *smem + tri_bytes, &with);
        if (e == cudaSuccess) e = trace_occupancy(adjoint, true, false, c->depth, *threads, *smem, &without);
        if (e != cudaSuccess) return cuda_fail(c, e, "occupancy query");
        const int want = c->blocks_per_sm > 0 ? std::min(c->blocks_per_sm, without) : without;
        tris = with >= std::max(want, 1);
    }
    p->n_tris_staged = tris ? c->n_tri : 0;
    if (tris) *smem += tri_bytes;
    int bps = c->blocks_per_sm;
    if (bps <= 0) {
        cudaError_t e = trace_occupancy(adjoint, staged, tris, c->depth, *threads, *smem, &bps);
        if (e != cudaSuccess) return cuda_fail(c, e, "occupancy query");
        if (bps < 1) return fail(c, LT_ERR_ARG, "launch shape does not fit on an SM");
    }
    *grid = c->sm_count * bps;
    return LT_OK;
}

// Upper bound on the step-loop iterations of a warp: every iteration
// advances at least one of its 32 lanes by one step, and a lane needs at most
// max_hits segments per photon, each at most max_steps + 1 node steps (the
// last one gives up), 8 leaf steps per node visited and one finish.
uint64_t step_limit(const TraceParams &p) {
    const uint64_t per_segment = (uint64_t)(kWide + 1) * (uint64_t)p.max_steps + 2;
    return 32ull * ((uint64_t)p.chunk * (uint64_t)p.max_hits * per_segment + 1);
}

uint64_t photon_chunk(uint64_t n, int grid, int threads) {
    const uint64_t T = (uint64_t)grid * (uint64_t)threads;
    return std::max<uint64_t>(1, (n + T - 1) / T);
}

TraceParams base_params(Ctx *c, uint64_t seed, int32_t max_hits, uint64_t begin, uint64_t end) {
    TraceParams p;
    std::memset(&p, 0, sizeof(p));
    p.nodes = c->d_nodes;
    p.cnodes = c->d_cnodes;
    p.parent = c->d_parent;
    p.n_nodes = c->n_nodes;
    p.depth = c->depth;
    p.tris = c->d_tris;
    p.hits = c->d_hits;
    p.lights = c->d_lights;
    p.n_lights = (int32_t)c->lights.size();
    p.max_hits = max_hits;
    p.max_steps = c->max_steps > 0 ? c->max_steps : 16 * c->n_nodes + 64;
    p.hdr = nullptr;
    p.seed = seed;
    p.photon_begin = begin;
    p.photon_end = end;
    p.n_texels = c->n_texels;
    p.err = c->d_err;
    return p;
}

int check_trace_args(Ctx *c, uint64_t n_photons, int32_t max_hits, uint64_t begin, uint64_t end) {
    if (!c->d_nodes) return fail(c, LT_ERR_STATE, "no scene uploaded");
    if (c->lights.empty()) return fail(c, LT_ERR_STATE, "no lights set");
    if (n_photons == 0) return fail(c, LT_ERR_ARG, "n_photons must be positive");
    if (max_hits < 1 || max_hits > 64) return fail(c, LT_ERR_ARG, "max_hits must be in [1, 64]");
    if (begin > end || end > n_photons) return fail(c, LT_ERR_ARG, "photon range outside [0, n_photons]");
    if (end - begin > kMaxPassPhotons) return fail(c, LT_ERR_ARG, "a pass covers at most 2^32 - 1 photons");
    return LT_OK;
}

// ---------------------------------------------------------------------------
// Batched designs
// ---------------------------------------------------------------------------
constexpr size_t kHdrBytes = 256;   // StepHeader, then the light records

void batch_drop_graph(Ctx *c) {
    if (c->batch.exec) cudaGraphExecDestroy(c->batch.exec);
    if (c->batch.graph) cudaGraphDestroy(c->batch.graph);
    c->batch.exec = nullptr;
    c->batch.graph = nullptr;
}

void batch_free(Ctx *c) {
    Ctx::Batch &b = c->batch;
    if (b.stream) cudaStreamSynchronize(b.stream);
    batch_drop_graph(c);
    dfree(b.d_in); dfree(b.d_q); dfree(b.d_E); dfree(b.d_w); dfree(b.d_partial); dfree(b.d_loss); dfree(b.d_grad);
    dfree(b.d_slots); dfree(b.d_gfix); dfree(b.d_gscale); dfree(b.d_wmax); dfree(b.d_gpart); dfree(b.d_rec);
    if (b.h_in) cudaFreeHost(b.h_in);
    if (b.h_out) cudaFreeHost(b.h_out);
    if (b.stream) cudaStreamDestroy(b.stream);
    b = Ctx::Batch();
}

struct BatchLaunch {
    TraceParams fwd, adj, grad;
    LossParams loss;
    int grid_f, grid_a, threads_f, threads_a;
    size_t smem_f, smem_a;
    int32_t grad_parts;
};

// Launch parameters of a batch step; grows the gradient slots if needed.
// Runs before any stream capture (it may allocate).
int batch_prepare(Ctx *c, BatchLaunch *bl) {
    Ctx::Batch &b = c->batch;
    const uint64_t n_total = b.photons * (uint64_t)b.n_designs;
    const StepHeader *hdr = reinterpret_cast<const StepHeader *>(b.d_in);
    const LightDev *lights = reinterpret_cast<const LightDev *>(b.d_in + kHdrBytes);
    int rc;
    bl->fwd = base_params(c, 0, b.max_hits, 0, n_total);
    bl->fwd.lights = lights;
    bl->fwd.n_lights = b.n_lights;
    bl->fwd.hdr = hdr;
    bl->fwd.q = b.d_q;
    bl->fwd.segments = reinterpret_cast<unsigned long long *>(b.d_grad + (size_t)b.n_lights * 8);
    if ((rc = launch_shape(c, false, &bl->grid_f, &bl->threads_f, &bl->smem_f, &bl->fwd))) return rc;
    bl->fwd.chunk = photon_chunk(n_total, bl->grid_f, bl->threads_f);
    bl->fwd.max_iters = step_limit(bl->fwd);
    bl->adj = bl->fwd;
    bl->adj.q = nullptr;
    bl->adj.w = b.d_w;
    bl->adj.wmax = b.d_wmax;
    bl->adj.segments = bl->fwd.segments + 1;
    if ((rc = launch_shape(c, true, &bl->grid_a, &bl->threads_a, &bl->smem_a, &bl->adj))) return rc;
    bl->adj.chunk = photon_chunk(n_total, bl->grid_a, bl->threads_a);
    bl->adj.max_iters = step_limit(bl->adj);
    int32_t max_count = 1, min_count = INT32_MAX;
    for (int32_t n : b.counts) {
        max_count = std::max(max_count, n);
        min_count = std::min(min_count, n);
    }
    bool grown = false;
    if ((rc = grow(c, b.d_rec, b.rec_bytes, (size_t)n_total * sizeof(PhotonAdj), b.stream, &grown))) return rc;
    bl->adj.rec_adj = b.d_rec;
    bl->grad = grad_params(bl->adj, b.photons / (uint64_t)max_count, nullptr, c->sm_count);
    if ((rc = grow(c, b.d_slots, b.slots_bytes, grad_slot_bytes(bl->grad), b.stream, &grown))) return rc;
    bl->grad.slots = b.d_slots;
    bl->grad_parts = grad_parts((b.photons + (uint64_t)min_count - 1) / (uint64_t)min_count, bl->grad.chunk);
    const size_t need_parts = (size_t)b.n_lights * (size_t)bl->grad_parts * 8 * sizeof(ulonglong2);
    if ((rc = grow(c, b.d_gpart, b.gpart_bytes, need_parts, b.stream, &grown))) return rc;
    if (grown) batch_drop_graph(c);     // a captured step holds the old buffers
    LossParams &lp = bl->loss;
    lp.q = b.d_q;
    lp.E_target = c->d_target;
    lp.alpha = c->has_alpha ? c->d_alpha : nullptr;
    lp.area = c->d_area;
    lp.inv_scale = 0.0;
    lp.hdr = hdr;
    lp.n_texels = c->n_texels;
    lp.n_designs = b.n_designs;
    lp.E_out = b.d_E;
    lp.w_out = b.d_w;
    lp.partial = b.d_partial;
    lp.loss_out = b.d_loss;
    return LT_OK;
}

// The work of one step, in stream order: lights and header in, forward,
// objective per design, adjoint, gradient sums, results out to pinned memory.
int batch_issue(Ctx *c, const BatchLaunch &bl) {
    Ctx::Batch &b = c->batch;
    const cudaStream_t s = b.stream;
    const size_t T = (size_t)c->n_texels, D = (size_t)b.n_designs, L = (size_t)b.n_lights;
    LT_CUDA(c, cudaMemcpyAsync(b.d_in, b.h_in, b.in_bytes, cudaMemcpyHostToDevice, s));
    LT_CUDA(c, cudaMemsetAsync(b.d_q, 0, D * T * sizeof(unsigned long long), s));
    LT_CUDA(c, cudaMemsetAsync(bl.fwd.segments, 0, 2 * sizeof(unsigned long long), s));
    LT_CUDA(c, launch_forward(bl.fwd, bl.grid_f, bl.threads_f, bl.smem_f, s));
    LT_CUDA(c, launch_loss(bl.loss, s));
    LT_CUDA(c, launch_weight_range(b.d_w, (int64_t)(D * T), b.d_wmax, s));
    LT_CUDA(c, launch_adjoint(bl.adj, bl.grid_a, bl.threads_a, bl.smem_a, s));
    LT_CUDA(c, launch_grad_photons(bl.grad, s));
    LT_CUDA(c, launch_grad_finalize(bl.grad, b.d_gpart, bl.grad_parts, b.d_grad, b.d_gfix, b.d_gscale, s));
    LT_CUDA(c, cudaMemcpyAsync(b.h_out, b.d_loss, D * sizeof(double), cudaMemcpyDeviceToHost, s));
    LT_CUDA(c, cudaMemcpyAsync(b.h_out + D, b.d_grad, (L * 8 + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
    return LT_OK;
}

int batch_check_device(Ctx *c) {
    int32_t e = 0;
    LT_CUDA(c, cudaMemcpyAsync(&e, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->batch.stream));
    LT_CUDA(c, cudaStreamSynchronize(c->batch.stream));
    if (e) {
        LT_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->batch.stream));
        LT_CUDA(c, cudaStreamSynchronize(c->batch.stream));
        return device_error(c, e);
    }
    return LT_OK;
}

}  // namespace

extern "C" {

int lt_version(void) { return 2; }

static_assert(sizeof(lt_bvh_node) == sizeof(Node), "lt_bvh_node mirrors lt::Node");
static_assert(offsetof(lt_bvh_node, hi_z) == offsetof(Node, hiz) && offsetof(lt_bvh_node, child) == offsetof(Node, child) &&
                  offsetof(lt_bvh_node, inner_mask) == offsetof(Node, inner_mask),
              "lt_bvh_node field offsets");

int lt_build_bvh(const float *tri_xyz, int32_t n_tri, lt_bvh_node *nodes_out, int32_t nodes_cap, int32_t *order_out,
                 int32_t *n_nodes_out, int32_t *depth_out) {
    LT_TRY
    if (!tri_xyz || n_tri <= 0) return LT_ERR_ARG;
    for (size_t k = 0; k < (size_t)n_tri * 9; ++k)
        if (!std::isfinite(tri_xyz[k])) return LT_ERR_ARG;
    BvhBuild bvh;
    std::string err;
    maybe_inject_host_oom();
    if (!build_wide_bvh(tri_xyz, n_tri, &bvh, &err)) return LT_ERR_ARG;
    const int32_t n_nodes = (int32_t)bvh.nodes.size();
    if (n_nodes_out) *n_nodes_out = n_nodes;
    if (depth_out) *depth_out = bvh.depth;
    if (nodes_out) {
        if (nodes_cap < n_nodes) return LT_ERR_ARG;
        std::memcpy(nodes_out, bvh.nodes.data(), sizeof(Node) * (size_t)n_nodes);
    }
    if (order_out) std::memcpy(order_out, bvh.order.data(), sizeof(int32_t) * (size_t)n_tri);
    return LT_OK;
    LT_CATCH(nullptr)
}

static_assert(sizeof(lt_bvh_cnode) == sizeof(CNode), "lt_bvh_cnode mirrors lt::CNode");
static_assert(offsetof(lt_bvh_cnode, meta) == offsetof(CNode, meta) && offsetof(lt_bvh_cnode, q) == offsetof(CNode, q) &&
                  offsetof(lt_bvh_cnode, child) == offsetof(CNode, child),
              "lt_bvh_cnode field offsets");

int lt_compress_bvh(const lt_bvh_node *nodes, int32_t n_nodes, lt_bvh_cnode *out) {
    LT_TRY
    if (!nodes || !out || n_nodes <= 0) return LT_ERR_ARG;
    const Node *in = reinterpret_cast<const Node *>(nodes);
    for (int32_t i = 0; i < n_nodes; ++i)
        for (int k = 0; k < kWide; ++k)
            if (in[i].child[k] != kEmptyChild &&
                !(std::isfinite(in[i].lox[k]) && std::isfinite(in[i].hix[k]) && std::isfinite(in[i].loy[k]) &&
                  std::isfinite(in[i].hiy[k]) && std::isfinite(in[i].loz[k]) && std::isfinite(in[i].hiz[k]) &&
                  in[i].lox[k] <= in[i].hix[k] && in[i].loy[k] <= in[i].hiy[k] && in[i].loz[k] <= in[i].hiz[k]))
                return LT_ERR_ARG;
    return compress_nodes(in, n_nodes, reinterpret_cast<CNode *>(out)) ? LT_OK : LT_ERR_ARG;
    LT_CATCH(nullptr)
}

int lt_create(void **ctx_out, int device, void *cuda_stream) {
    LT_TRY
    if (!ctx_out) return LT_ERR_ARG;
    *ctx_out = nullptr;
    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return LT_ERR_OOM;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || device < 0 || device >= n_dev) {
        delete c;
        return e != cudaSuccess ? LT_ERR_CUDA : LT_ERR_ARG;
    }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&c->d_seg, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_loss, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_partial, kLossBlocks * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_pinned, 64 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_lights, LT_MAX_LIGHTS * sizeof(LightDev)) != cudaSuccess ||
        cudaMallocHost(&c->h_lights, LT_MAX_LIGHTS * sizeof(LightDev)) != cudaSuccess ||
        cudaMalloc(&c->d_grad, LT_MAX_LIGHTS * 8 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_gfix, LT_MAX_LIGHTS * 8 * sizeof(ulonglong2)) != cudaSuccess ||
        cudaMalloc(&c->d_gscale, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_wmax, sizeof(uint32_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->lights_copied, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(c->lights_copied, c->stream) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(c->d_seg, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        lt_destroy(c);
        return LT_ERR_CUDA;
    }
    *ctx_out = c;
    return LT_OK;
    LT_CATCH(nullptr)
}

int lt_destroy(void *ctx) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    dfree(c->d_nodes); dfree(c->d_cnodes); dfree(c->d_parent); dfree(c->d_tris); dfree(c->d_hits); dfree(c->d_area);
    dfree(c->d_target); dfree(c->d_alpha); dfree(c->d_lights); dfree(c->d_q); dfree(c->d_E); dfree(c->d_w);
    dfree(c->d_loss); dfree(c->d_partial); dfree(c->d_grad); dfree(c->d_slots); dfree(c->d_seg);
    dfree(c->d_err); dfree(c->d_gfix); dfree(c->d_gscale); dfree(c->d_wmax); dfree(c->d_gpart); dfree(c->d_rec);
    batch_free(c);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->h_lights) cudaFreeHost(c->h_lights);
    if (c->lights_copied) cudaEventDestroy(c->lights_copied);
    delete c;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_set_stream(void *ctx, void *cuda_stream) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return LT_OK;
    LT_CATCH(ctx)
}

const char *lt_last_error(const void *ctx) {
    const Ctx *c = static_cast<const Ctx *>(ctx);
    return c ? c->err.c_str() : "null context";
}

int lt_upload_scene(void *ctx, const float *tri_xyz, const float *tri_uv, const int32_t *tri_tile,
                    const float *tri_albedo, int32_t n_tri, const int32_t *tile_res, const double *tile_area,
                    int32_t n_tiles, int64_t *n_texels_out) {
    LT_TRY
    NvtxRange nvtx_range("lt_upload_scene");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!tri_xyz || !tri_uv || !tri_tile || !tri_albedo || !tile_res || !tile_area || n_tri <= 0 || n_tiles <= 0)
        return fail(c, LT_ERR_ARG, "null scene array or empty scene");
    LT_CUDA(c, cudaSetDevice(c->device));
    std::vector<int64_t> off((size_t)n_tiles + 1, 0);
    for (int32_t k = 0; k < n_tiles; ++k) {
        const int32_t ru = tile_res[2 * k], rv = tile_res[2 * k + 1];
        if (ru < 1 || rv < 1) return fail(c, LT_ERR_ARG, "tile resolution must be >= 1");
        if (!(tile_area[k] > 0.0) || !std::isfinite(tile_area[k])) return fail(c, LT_ERR_ARG, "tile area must be > 0");
        off[k + 1] = off[k] + (int64_t)ru * rv;
    }
    for (int32_t i = 0; i < n_tri; ++i) {
        if (tri_tile[i] < 0 || tri_tile[i] >= n_tiles) return fail(c, LT_ERR_ARG, "triangle tile out of range");
        if (!(tri_albedo[i] >= 0.0f && tri_albedo[i] <= 1.0f)) return fail(c, LT_ERR_ARG, "albedo must be in [0, 1]");
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(tri_xyz[9 * (size_t)i + k])) return fail(c, LT_ERR_ARG, "non-finite vertex");
    }
    BvhBuild bvh;
    std::string berr;
    maybe_inject_host_oom();
    if (!build_wide_bvh(tri_xyz, n_tri, &bvh, &berr)) return fail(c, LT_ERR_ARG, berr);
    std::vector<CNode> cnodes(bvh.nodes.size());
    if (!compress_nodes(bvh.nodes.data(), (int32_t)bvh.nodes.size(), cnodes.data()))
        return fail(c, LT_ERR_ARG, "a BVH node wider than about 2e6: beyond the range of the compressed nodes");
    std::vector<Tri> tris((size_t)n_tri);
    std::vector<TriHit> hits((size_t)n_tri);
    for (int32_t j = 0; j < n_tri; ++j) {
        const int32_t i = bvh.order[j];
        Tri &t = tris[j];
        const float *v = tri_xyz + 9 * (size_t)i;
        for (int k = 0; k < 3; ++k) { t.v0[k] = v[k]; t.v1[k] = v[3 + k]; t.v2[k] = v[6 + k]; }
        t.prim = i;
        t.tile = tri_tile[i];
        t.albedo = tri_albedo[i];
        TriHit &h = hits[j];
        for (int k = 0; k < 6; ++k) h.uv[k] = tri_uv[6 * (size_t)i + k];
        h.res_u = tile_res[2 * tri_tile[i]];
        h.res_v = tile_res[2 * tri_tile[i] + 1];
        h.texel_off = off[tri_tile[i]];
        double e1[3], e2[3], nn[3];
        for (int k = 0; k < 3; ++k) { e1[k] = (double)v[3 + k] - v[k]; e2[k] = (double)v[6 + k] - v[k]; }
        nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double ln = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        if (!(ln > 0.0)) return fail(c, LT_ERR_ARG, "degenerate triangle " + std::to_string(i));
        for (int k = 0; k < 3; ++k) h.n[k] = (float)(nn[k] / ln);
        for (int k = 0; k < 3; ++k) h.pad[k] = 0.0f;
    }
    const int64_t T = off[n_tiles];
    c->h_xyz.assign(tri_xyz, tri_xyz + 9 * (size_t)n_tri);
    c->h_uv.assign(tri_uv, tri_uv + 6 * (size_t)n_tri);
    c->h_tile.assign(tri_tile, tri_tile + n_tri);
    c->h_res.assign(tile_res, tile_res + 2 * (size_t)n_tiles);
    c->h_off = off;
    std::vector<float> area((size_t)T);
    for (int32_t k = 0; k < n_tiles; ++k) {
        const float a = (float)(tile_area[k] / ((double)tile_res[2 * k] * (double)tile_res[2 * k + 1]));
        std::fill(area.begin() + off[k], area.begin() + off[k + 1], a);
    }
    LT_CUDA(c, cudaStreamSynchronize(c->stream));
    batch_free(c);     // batch buffers are sized by the old texel count
    LT_CUDA(c, dalloc(c->d_nodes, bvh.nodes.size()));
    LT_CUDA(c, dalloc(c->d_cnodes, cnodes.size()));
    LT_CUDA(c, dalloc(c->d_parent, bvh.parent.size()));
    LT_CUDA(c, dalloc(c->d_tris, (size_t)n_tri));
    LT_CUDA(c, dalloc(c->d_hits, (size_t)n_tri));
    LT_CUDA(c, dalloc(c->d_area, (size_t)T));
    LT_CUDA(c, dalloc(c->d_q, (size_t)T));
    LT_CUDA(c, dalloc(c->d_E, (size_t)T));
    LT_CUDA(c, dalloc(c->d_w, (size_t)T));
    LT_CUDA(c, dalloc(c->d_target, (size_t)T));
    dfree(c->d_alpha);
    LT_CUDA(c, cudaMemcpy(c->d_nodes, bvh.nodes.data(), bvh.nodes.size() * sizeof(Node), cudaMemcpyHostToDevice));
    LT_CUDA(c, cudaMemcpy(c->d_cnodes, cnodes.data(), cnodes.size() * sizeof(CNode), cudaMemcpyHostToDevice));
    LT_CUDA(c, cudaMemcpy(c->d_parent, bvh.parent.data(), bvh.parent.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice));
    LT_CUDA(c, cudaMemcpy(c->d_tris, tris.data(), tris.size() * sizeof(Tri), cudaMemcpyHostToDevice));
    LT_CUDA(c, cudaMemcpy(c->d_hits, hits.data(), hits.size() * sizeof(TriHit), cudaMemcpyHostToDevice));
    LT_CUDA(c, cudaMemcpy(c->d_area, area.data(), area.size() * sizeof(float), cudaMemcpyHostToDevice));
    LT_CUDA(c, cudaMemset(c->d_target, 0, (size_t)T * sizeof(float)));
    c->n_nodes = (int32_t)bvh.nodes.size();
    c->n_tri = n_tri;
    c->depth = bvh.depth;
    c->n_texels = T;
    c->fwd_done = c->has_w = c->has_target = c->has_alpha = false;
    c->stats = lt_stats{};
    c->stats.n_texels = T;
    c->stats.n_triangles = n_tri;
    c->stats.n_nodes = c->n_nodes;
    c->stats.bvh_depth = c->depth;
    if (n_texels_out) *n_texels_out = T;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_set_target(void *ctx, const float *E_target, const float *alpha, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!c->d_nodes) return fail(c, LT_ERR_STATE, "no scene uploaded");
    if (!E_target) return fail(c, LT_ERR_ARG, "null target");
    int rc = copy_in(c, c->d_target, E_target, (size_t)c->n_texels * sizeof(float), is_device);
    if (rc) return rc;
    if (alpha) {
        if (!c->d_alpha) LT_CUDA(c, dalloc(c->d_alpha, (size_t)c->n_texels));
        rc = copy_in(c, c->d_alpha, alpha, (size_t)c->n_texels * sizeof(float), is_device);
        if (rc) return rc;
        c->has_alpha = true;
    } else {
        c->has_alpha = false;
    }
    if (!is_device) LT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_target = true;
    return LT_OK;
    LT_CATCH(ctx)
}

// Argument checks of one luminaire; empty on success.
static const char *light_error(const lt_light &s) {
    if (s.type != LT_POINT && s.type != LT_SPOT && s.type != LT_AREA) return "unknown light type";
    bool finite = std::isfinite(s.p_int) && std::isfinite(s.yaw) && std::isfinite(s.pitch);
    for (int k = 0; k < 3; ++k) finite = finite && std::isfinite(s.pos[k]);
    if (!finite) return "non-finite light parameter";
    if (s.type == LT_SPOT && !(s.theta_in >= 0.0f && s.theta_in < s.theta_out && s.theta_out <= (float)kPi))
        return "spot cone needs 0 <= theta_in < theta_out <= pi";
    if (s.type == LT_AREA && !(s.theta_in > 0.0f && s.theta_out > 0.0f && std::isfinite(s.theta_in) &&
                               std::isfinite(s.theta_out)))
        return "area light needs a positive finite width and height";
    return nullptr;
}

int lt_set_lights(void *ctx, const lt_light *lights, int32_t n_lights) {
    LT_TRY
    NvtxRange nvtx_range("lt_set_lights");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!lights || n_lights < 1 || n_lights > LT_MAX_LIGHTS) return fail(c, LT_ERR_ARG, "n_lights out of range");
    for (int32_t l = 0; l < n_lights; ++l)
        if (const char *e = light_error(lights[l])) return fail(c, LT_ERR_ARG, e);
    c->lights.assign(lights, lights + n_lights);
    c->lights_dirty = true;
    return LT_OK;
    LT_CATCH(ctx)
}

// Fixed point: S = 2^k with S * (total power bound) * max_hits < 2^62, so
// no texel (nor the sum of all texels) can overflow int64. Returns false
// when k would fall below -120 (a power bound beyond 2^182 / max_hits): the
// float deposit Phi * S would then lose its precision.
static bool fixed_point_scale(double bound, int32_t max_hits, double *S) {
    *S = std::ldexp(1.0, 40);
    if (!(bound > 0.0)) return true;
    if (!std::isfinite(bound)) return false;
    const int k = (int)std::floor(std::log2(std::ldexp(1.0, 62) / (bound * (double)max_hits)));
    if (k < -120) return false;
    *S = std::ldexp(1.0, std::min(120, k));
    return true;
}

static int forward_pass(Ctx *c, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                 uint64_t photon_end, unsigned long long *d_work) {
    int rc = check_trace_args(c, n_photons, max_hits, photon_begin, photon_end);
    if (rc) return rc;
    LT_CUDA(c, cudaSetDevice(c->device));
    if ((rc = upload_lights(c, n_photons))) return rc;
    double S;
    if (!fixed_point_scale(c->power_bound, max_hits, &S))
        return fail(c, LT_ERR_OVERFLOW, "total light power too large for the int64 texel accumulator");
    c->scale = S;
    TraceParams p = base_params(c, seed, max_hits, photon_begin, photon_end);
    p.q = c->d_q;
    p.scale = (float)S;
    p.segments = c->d_seg;
    int grid, threads;
    size_t smem;
    if ((rc = launch_shape(c, false, &grid, &threads, &smem, &p))) return rc;
    p.chunk = photon_chunk(photon_end - photon_begin, grid, threads);
    p.max_iters = step_limit(p);
    LT_CUDA(c, cudaMemsetAsync(c->d_q, 0, (size_t)c->n_texels * sizeof(unsigned long long), c->stream));
    LT_CUDA(c, cudaMemsetAsync(c->d_seg, 0, sizeof(unsigned long long), c->stream));
    if (d_work) {
        p.work = d_work;
        LT_CUDA(c, launch_forward_counted(p, grid, threads, smem, c->stream));
    } else {
        LT_CUDA(c, launch_forward(p, grid, threads, smem, c->stream));
    }
    c->fwd_done = true;
    c->has_w = false;
    c->seg_single = true;
    c->stats.photons_forward = photon_end - photon_begin;
    c->stats.staged_nodes = p.n_staged;
    c->stats.staged_triangles = p.n_tris_staged;
    c->stats.fixed_point_scale = S;
    c->stats.grid_blocks = grid;
    c->stats.block_threads = threads;
    return LT_OK;
}

int lt_trace_forward(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                     uint64_t photon_end) {
    LT_TRY
    NvtxRange nvtx_range("lt_trace_forward");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    return forward_pass(c, seed, n_photons, max_hits, photon_begin, photon_end, nullptr);
    LT_CATCH(ctx)
}

int lt_count_work(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                  uint64_t photon_end, uint64_t *counts_out) {
    LT_TRY
    NvtxRange nvtx_range("lt_count_work");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!counts_out) return fail(c, LT_ERR_ARG, "null counts output");
    unsigned long long *d_work = nullptr;
    LT_CUDA(c, cudaSetDevice(c->device));
    LT_CUDA(c, cudaMalloc(&d_work, 2 * sizeof(unsigned long long)));
    cudaError_t e = cudaMemsetAsync(d_work, 0, 2 * sizeof(unsigned long long), c->stream);
    int rc = e == cudaSuccess ? forward_pass(c, seed, n_photons, max_hits, photon_begin, photon_end, d_work)
                              : cuda_fail(c, e, "cudaMemsetAsync");
    unsigned long long h[3] = {0, 0, 0};
    if (rc == LT_OK) {
        e = cudaMemcpyAsync(h, d_work, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h + 2, c->d_seg, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                                  c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "lt_count_work");
    }
    cudaFree(d_work);
    if (rc) return rc;
    counts_out[0] = h[2];
    counts_out[1] = h[0];
    counts_out[2] = h[1];
    counts_out[3] = photon_end - photon_begin;
    return check_device(c);
    LT_CATCH(ctx)
}

int lt_texel_accumulator(void *ctx, int64_t **q_device, double *scale_out) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !q_device) return LT_ERR_ARG;
    if (!c->d_q) return fail(c, LT_ERR_STATE, "no scene uploaded");
    *q_device = reinterpret_cast<int64_t *>(c->d_q);
    if (scale_out) *scale_out = c->scale;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_get_texel_sums(void *ctx, int64_t *q_out, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !q_out) return LT_ERR_ARG;
    if (!c->fwd_done) return fail(c, LT_ERR_STATE, "no forward pass");
    LT_CUDA(c, cudaSetDevice(c->device));
    return copy_out(c, q_out, c->d_q, (size_t)c->n_texels * sizeof(int64_t), is_device);
    LT_CATCH(ctx)
}

int lt_loss(void *ctx, double *loss_out, int is_device) {
    LT_TRY
    NvtxRange nvtx_range("lt_loss");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!c->fwd_done) return fail(c, LT_ERR_STATE, "lt_loss needs a forward pass");
    if (!c->has_target) return fail(c, LT_ERR_STATE, "lt_loss needs a target (lt_set_target)");
    LT_CUDA(c, cudaSetDevice(c->device));
    LossParams p;
    p.q = c->d_q;
    p.E_target = c->d_target;
    p.alpha = c->has_alpha ? c->d_alpha : nullptr;
    p.area = c->d_area;
    p.inv_scale = 1.0 / c->scale;
    p.hdr = nullptr;
    p.n_texels = c->n_texels;
    p.n_designs = 1;
    p.E_out = c->d_E;
    p.w_out = c->d_w;
    p.partial = c->d_partial;
    p.loss_out = c->d_loss;
    LT_CUDA(c, launch_loss(p, c->stream));
    c->has_w = true;
    if (loss_out) {
        int rc = copy_out(c, loss_out, c->d_loss, sizeof(double), is_device);
        if (rc) return rc;
        if (!is_device) return check_device(c);
    }
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_get_irradiance(void *ctx, float *E_out, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !E_out) return LT_ERR_ARG;
    if (!c->fwd_done) return fail(c, LT_ERR_STATE, "no forward pass");
    LT_CUDA(c, cudaSetDevice(c->device));
    LT_CUDA(c, launch_resolve(c->d_q, c->d_area, 1.0 / c->scale, c->n_texels, c->d_E, c->stream));
    return copy_out(c, E_out, c->d_E, (size_t)c->n_texels * sizeof(float), is_device);
    LT_CATCH(ctx)
}

int lt_texel_areas(void *ctx, float *A_out, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !A_out) return LT_ERR_ARG;
    if (!c->d_area) return fail(c, LT_ERR_STATE, "no scene uploaded");
    LT_CUDA(c, cudaSetDevice(c->device));
    return copy_out(c, A_out, c->d_area, (size_t)c->n_texels * sizeof(float), is_device);
    LT_CATCH(ctx)
}

int lt_set_adjoint_weights(void *ctx, const float *w, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !w) return LT_ERR_ARG;
    if (!c->d_w) return fail(c, LT_ERR_STATE, "no scene uploaded");
    LT_CUDA(c, cudaSetDevice(c->device));
    int rc = copy_in(c, c->d_w, w, (size_t)c->n_texels * sizeof(float), is_device);
    if (rc) return rc;
    if (!is_device) LT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_w = true;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_trace_adjoint(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                     uint64_t photon_end, double *grad_out, int is_device) {
    LT_TRY
    NvtxRange nvtx_range("lt_trace_adjoint");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!grad_out) return fail(c, LT_ERR_ARG, "null gradient output");
    int rc = check_trace_args(c, n_photons, max_hits, photon_begin, photon_end);
    if (rc) return rc;
    if (!c->has_w) return fail(c, LT_ERR_STATE, "lt_trace_adjoint needs weights (lt_loss or lt_set_adjoint_weights)");
    LT_CUDA(c, cudaSetDevice(c->device));
    if ((rc = upload_lights(c, n_photons))) return rc;
    const int32_t L = (int32_t)c->lights.size();
    TraceParams p = base_params(c, seed, max_hits, photon_begin, photon_end);
    p.w = c->d_w;
    p.wmax = c->d_wmax;
    p.flux_max = c->flux_max;
    p.segments = c->d_seg + 1;
    int grid, threads;
    size_t smem;
    if ((rc = launch_shape(c, true, &grid, &threads, &smem, &p))) return rc;
    p.chunk = photon_chunk(photon_end - photon_begin, grid, threads);
    p.max_iters = step_limit(p);
    if ((rc = grow(c, c->d_rec, c->rec_bytes, (size_t)(photon_end - photon_begin) * sizeof(PhotonAdj), c->stream)))
        return rc;
    p.rec_adj = c->d_rec;
    TraceParams pg = grad_params(p, n_photons / (uint64_t)L, nullptr, c->sm_count);
    if ((rc = grow(c, c->d_slots, c->slots_bytes, grad_slot_bytes(pg), c->stream))) return rc;
    pg.slots = c->d_slots;
    const int32_t parts = grad_parts((n_photons + (uint64_t)L - 1) / (uint64_t)L, pg.chunk);
    const size_t need_parts = (size_t)L * (size_t)parts * 8 * sizeof(ulonglong2);
    if ((rc = grow(c, c->d_gpart, c->gpart_bytes, need_parts, c->stream))) return rc;
    LT_CUDA(c, cudaMemsetAsync(c->d_seg + 1, 0, sizeof(unsigned long long), c->stream));
    LT_CUDA(c, launch_weight_range(c->d_w, c->n_texels, c->d_wmax, c->stream));
    LT_CUDA(c, launch_adjoint(p, grid, threads, smem, c->stream));
    LT_CUDA(c, launch_grad_photons(pg, c->stream));
    LT_CUDA(c, launch_grad_finalize(pg, c->d_gpart, parts, c->d_grad, c->d_gfix, c->d_gscale, c->stream));
    c->adj_lights = L;
    c->stats.photons_adjoint = photon_end - photon_begin;
    c->seg_single = true;
    rc = copy_out(c, grad_out, c->d_grad, (size_t)L * 8 * sizeof(double), is_device);
    if (rc) return rc;
    if (!is_device) return check_device(c);
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_gradient_fixed(void *ctx, int64_t *sums_out, double *scale_out) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!sums_out || !scale_out) return fail(c, LT_ERR_ARG, "null output");
    if (!c->adj_lights) return fail(c, LT_ERR_STATE, "no adjoint pass");
    LT_CUDA(c, cudaSetDevice(c->device));
    LT_CUDA(c, cudaMemcpyAsync(sums_out, c->d_gfix, (size_t)c->adj_lights * 8 * sizeof(ulonglong2),
                               cudaMemcpyDeviceToHost, c->stream));
    LT_CUDA(c, cudaMemcpyAsync(scale_out, c->d_gscale, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LT_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_device(c);
    LT_CATCH(ctx)
}

int lt_debug_paths(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                   uint64_t count, int32_t *tri_out, int64_t *texel_out, double *grad_out) {
    LT_TRY
    NvtxRange nvtx_range("lt_debug_paths");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!tri_out || !texel_out) return fail(c, LT_ERR_ARG, "null output");
    int rc = check_trace_args(c, n_photons, max_hits, photon_begin, photon_begin + count);
    if (rc) return rc;
    if (grad_out && !c->has_w) return fail(c, LT_ERR_STATE, "per-photon gradients need adjoint weights");
    if (count == 0) return LT_OK;
    LT_CUDA(c, cudaSetDevice(c->device));
    if ((rc = upload_lights(c, n_photons))) return rc;
    const size_t n = (size_t)count * (size_t)max_hits;
    int32_t *d_tri = nullptr;
    int64_t *d_tex = nullptr;
    double *d_grad = nullptr;
    cudaError_t e = cudaMalloc(&d_tri, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_tex, n * sizeof(int64_t));
    if (e == cudaSuccess && grad_out) e = cudaMalloc(&d_grad, (size_t)count * 8 * sizeof(double));
    if (e == cudaSuccess) {
        TraceParams p = base_params(c, seed, max_hits, photon_begin, photon_begin + count);
        p.rec_tri = d_tri;
        p.rec_texel = d_tex;
        p.rec_grad = d_grad;
        p.w = c->d_w;
        e = launch_paths(p, count, c->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(tri_out, d_tri, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(texel_out, d_tex, n * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, d_grad, (size_t)count * 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_tri);
    cudaFree(d_tex);
    cudaFree(d_grad);
    if (e != cudaSuccess) return cuda_fail(c, e, "lt_debug_paths");
    return check_device(c);
    LT_CATCH(ctx)
}

int lt_get_stats(void *ctx, lt_stats *out) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !out) return LT_ERR_ARG;
    LT_CUDA(c, cudaSetDevice(c->device));
    if (c->seg_single) {   // a batch step stores its counts when it returns
        unsigned long long seg[2] = {0, 0};
        LT_CUDA(c, cudaMemcpyAsync(seg, c->d_seg, sizeof(seg), cudaMemcpyDeviceToHost, c->stream));
        LT_CUDA(c, cudaStreamSynchronize(c->stream));
        c->stats.segments_forward = seg[0];
        c->stats.segments_adjoint = seg[1];
    }
    *out = c->stats;
    return check_device(c);
    LT_CATCH(ctx)
}

int lt_set_design(void *ctx, uint32_t design) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    c->design_word = design;
    c->lights_dirty = true;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_batch_setup(void *ctx, int32_t n_designs, const int32_t *lights_per_design, uint64_t photons_per_design,
                   int32_t max_hits) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!c->d_nodes) return fail(c, LT_ERR_STATE, "no scene uploaded");
    if (n_designs < 1 || !lights_per_design) return fail(c, LT_ERR_ARG, "need at least one design");
    if (photons_per_design == 0) return fail(c, LT_ERR_ARG, "photons_per_design must be positive");
    if (photons_per_design > kMaxPassPhotons / (uint64_t)n_designs)
        return fail(c, LT_ERR_ARG, "a batch pass covers at most 2^32 - 1 photons (designs x photons per design)");
    if (max_hits < 1 || max_hits > 64) return fail(c, LT_ERR_ARG, "max_hits must be in [1, 64]");
    int64_t total = 0;
    for (int32_t d = 0; d < n_designs; ++d) {
        if (lights_per_design[d] < 1) return fail(c, LT_ERR_ARG, "every design needs at least one light");
        total += lights_per_design[d];
    }
    if (total > LT_MAX_BATCH_LIGHTS) return fail(c, LT_ERR_ARG, "more lights than LT_MAX_BATCH_LIGHTS");
    LT_CUDA(c, cudaSetDevice(c->device));
    batch_free(c);
    Ctx::Batch &b = c->batch;
    b.n_designs = n_designs;
    b.n_lights = (int32_t)total;
    b.max_hits = max_hits;
    b.photons = photons_per_design;
    b.counts.assign(lights_per_design, lights_per_design + n_designs);
    b.in_bytes = kHdrBytes + sizeof(LightDev) * (size_t)total;
    const size_t DT = (size_t)n_designs * (size_t)c->n_texels;
    cudaError_t e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_in, b.in_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_in, b.in_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_out, ((size_t)n_designs + (size_t)total * 8 + 2) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_q, DT * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_E, DT * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_w, DT * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_partial, (size_t)n_designs * kLossBlocksBatch * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_loss, (size_t)n_designs * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_grad, ((size_t)total * 8 + 2) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_gfix, (size_t)total * 8 * sizeof(ulonglong2));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_gscale, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_wmax, sizeof(uint32_t));
    if (e != cudaSuccess) {
        batch_free(c);
        return cuda_fail(c, e, "lt_batch_setup");
    }
    std::memset(b.h_in, 0, b.in_bytes);
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_batch_set_lights(void *ctx, const lt_light *lights) {
    LT_TRY
    NvtxRange nvtx_range("lt_batch_set_lights");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    Ctx::Batch &b = c->batch;
    if (!b.n_designs) return fail(c, LT_ERR_STATE, "lt_batch_setup first");
    if (!lights) return fail(c, LT_ERR_ARG, "null lights");
    for (int32_t l = 0; l < b.n_lights; ++l)
        if (const char *e = light_error(lights[l])) return fail(c, LT_ERR_ARG, e);
    b.lights.assign(lights, lights + b.n_lights);
    LightDev *out = reinterpret_cast<LightDev *>(b.h_in + kHdrBytes);
    double bound = 0.0;
    int32_t off = 0;
    for (int32_t d = 0; d < b.n_designs; ++d) {
        bound = std::max(bound, derive_lights(lights + off, b.counts[d], b.photons, (uint64_t)d * b.photons,
                                              (uint64_t)d * (uint64_t)c->n_texels, (uint32_t)d, out + off));
        off += b.counts[d];
    }
    // one fixed-point scale for the batch, safe for its brightest design
    double S;
    if (!fixed_point_scale(bound, b.max_hits, &S))
        return fail(c, LT_ERR_OVERFLOW, "total light power too large for the int64 texel accumulator");
    StepHeader *h = reinterpret_cast<StepHeader *>(b.h_in);
    h->scale = S;
    h->inv_scale = 1.0 / S;
    h->flux_max = max_flux(out, b.n_lights);
    b.has_lights = true;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_batch_step(void *ctx, uint64_t seed_fwd, uint64_t seed_adj, double *loss_out, double *grad_out,
                  int use_graph) {
    LT_TRY
    NvtxRange nvtx_range("lt_batch_step");
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    Ctx::Batch &b = c->batch;
    if (!b.n_designs || !b.has_lights) return fail(c, LT_ERR_STATE, "lt_batch_setup and lt_batch_set_lights first");
    if (!c->has_target) return fail(c, LT_ERR_STATE, "no target (lt_set_target)");
    LT_CUDA(c, cudaSetDevice(c->device));
    StepHeader *h = reinterpret_cast<StepHeader *>(b.h_in);
    h->seed_fwd = seed_fwd;
    h->seed_adj = seed_adj;
    BatchLaunch bl;
    int rc = batch_prepare(c, &bl);
    if (rc) return rc;
    if (use_graph) {
        if (!b.exec) {
            LT_CUDA(c, cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeRelaxed));
            rc = batch_issue(c, bl);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b.stream, &g);
            if (rc || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return rc ? rc : cuda_fail(c, e, "cudaStreamEndCapture");
            }
            b.graph = g;
            const cudaError_t ei = cudaGraphInstantiate(&b.exec, b.graph, 0);
            if (ei != cudaSuccess) {
                batch_drop_graph(c);
                return cuda_fail(c, ei, "cudaGraphInstantiate");
            }
        }
        LT_CUDA(c, cudaGraphLaunch(b.exec, b.stream));
    } else {
        if ((rc = batch_issue(c, bl))) return rc;
    }
    LT_CUDA(c, cudaStreamSynchronize(b.stream));
    if ((rc = batch_check_device(c))) return rc;
    const size_t D = (size_t)b.n_designs, L = (size_t)b.n_lights;
    if (loss_out) std::memcpy(loss_out, b.h_out, D * sizeof(double));
    if (grad_out) std::memcpy(grad_out, b.h_out + D, L * 8 * sizeof(double));
    uint64_t seg[2];
    std::memcpy(seg, b.h_out + D + L * 8, sizeof(seg));
    b.segments = seg[0] + seg[1];
    c->stats.segments_forward = seg[0];
    c->stats.segments_adjoint = seg[1];
    c->stats.photons_forward = c->stats.photons_adjoint = b.photons * D;
    c->stats.fixed_point_scale = h->scale;
    c->stats.grid_blocks = bl.grid_f;
    c->stats.block_threads = bl.threads_f;
    c->stats.staged_nodes = bl.fwd.n_staged;
    c->stats.staged_triangles = bl.fwd.n_tris_staged;
    c->seg_single = false;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_texel_centres(void *ctx, float *pos_out, float *normal_out) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !pos_out || !normal_out) return LT_ERR_ARG;
    if (c->h_off.empty()) return fail(c, LT_ERR_STATE, "no scene uploaded");
    const int32_t n_tiles = (int32_t)c->h_res.size() / 2;
    std::vector<std::vector<int32_t>> tris_of((size_t)n_tiles);
    for (size_t i = 0; i < c->h_tile.size(); ++i) tris_of[(size_t)c->h_tile[i]].push_back((int32_t)i);
    for (int32_t k = 0; k < n_tiles; ++k) {
        const int32_t ru = c->h_res[2 * k], rv = c->h_res[2 * k + 1];
        for (int32_t j = 0; j < rv; ++j)
            for (int32_t i = 0; i < ru; ++i) {
                const double qu = (i + 0.5) / ru, qv = (j + 0.5) / rv;
                double best = -1e300, bp[3] = {0, 0, 0}, bn[3] = {0, 0, 1};
                for (int32_t tri : tris_of[(size_t)k]) {
                    const float *uv = c->h_uv.data() + 6 * (size_t)tri;
                    const float *X = c->h_xyz.data() + 9 * (size_t)tri;
                    // barycentric coordinates of (qu, qv) in the triangle's chart
                    const double e1u = (double)uv[2] - uv[0], e1v = (double)uv[3] - uv[1];
                    const double e2u = (double)uv[4] - uv[0], e2v = (double)uv[5] - uv[1];
                    const double det = e1u * e2v - e1v * e2u;
                    if (det == 0.0) continue;
                    const double du = qu - uv[0], dv = qv - uv[1];
                    double b1 = (du * e2v - dv * e2u) / det;
                    double b2 = (e1u * dv - e1v * du) / det;
                    double b0 = 1.0 - b1 - b2;
                    const double score = std::min(b0, std::min(b1, b2));
                    if (!(score > best)) continue;
                    best = score;
                    b0 = std::max(b0, 0.0);
                    b1 = std::max(b1, 0.0);
                    b2 = std::max(b2, 0.0);
                    const double sb = b0 + b1 + b2;
                    double e[2][3];
                    for (int a = 0; a < 3; ++a) {
                        bp[a] = (b0 * X[a] + b1 * X[3 + a] + b2 * X[6 + a]) / sb;
                        e[0][a] = (double)X[3 + a] - X[a];
                        e[1][a] = (double)X[6 + a] - X[a];
                    }
                    bn[0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
                    bn[1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
                    bn[2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
                    const double ln = std::sqrt(bn[0] * bn[0] + bn[1] * bn[1] + bn[2] * bn[2]);
                    for (int a = 0; a < 3; ++a) bn[a] /= ln;
                }
                const size_t t = (size_t)(c->h_off[k] + i + (int64_t)ru * j);
                for (int a = 0; a < 3; ++a) {
                    pos_out[3 * t + a] = (float)bp[a];
                    normal_out[3 * t + a] = (float)bn[a];
                }
            }
    }
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_batch_stream(void *ctx, void **stream_out) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !stream_out) return LT_ERR_ARG;
    *stream_out = (void *)c->batch.stream;
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_batch_texel_sums(void *ctx, int32_t design, int64_t *q_out, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !q_out) return LT_ERR_ARG;
    Ctx::Batch &b = c->batch;
    if (design < 0 || design >= b.n_designs) return fail(c, LT_ERR_ARG, "design out of range");
    LT_CUDA(c, cudaSetDevice(c->device));
    const size_t T = (size_t)c->n_texels;
    LT_CUDA(c, cudaMemcpyAsync(q_out, b.d_q + (size_t)design * T, T * sizeof(int64_t),
                               is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b.stream));
    LT_CUDA(c, cudaStreamSynchronize(b.stream));
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_batch_irradiance(void *ctx, int32_t design, float *E_out, int is_device) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !E_out) return LT_ERR_ARG;
    Ctx::Batch &b = c->batch;
    if (design < 0 || design >= b.n_designs) return fail(c, LT_ERR_ARG, "design out of range");
    LT_CUDA(c, cudaSetDevice(c->device));
    const size_t T = (size_t)c->n_texels;
    LT_CUDA(c, cudaMemcpyAsync(E_out, b.d_E + (size_t)design * T, T * sizeof(float),
                               is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b.stream));
    LT_CUDA(c, cudaStreamSynchronize(b.stream));
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_set_launch(void *ctx, int32_t threads_per_block, int32_t blocks_per_sm, int32_t smem_node_bytes) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (threads_per_block > 0 &&
        (threads_per_block % 32 || threads_per_block > std::max(trace_kernel_max_threads(true),
                                                                 trace_kernel_max_threads(false))))
        return fail(c, LT_ERR_ARG, "threads_per_block must be a multiple of 32 within the kernels' bounds");
    if (smem_node_bytes > 200 * 1024) return fail(c, LT_ERR_ARG, "smem_node_bytes must be in [0, 200 KiB]");
    if (threads_per_block >= 0) c->threads = threads_per_block;
    if (blocks_per_sm >= 0) c->blocks_per_sm = blocks_per_sm;
    if (smem_node_bytes >= 0) c->smem_node_bytes = smem_node_bytes;
    batch_drop_graph(c);     // a captured batch step holds the old launch shape
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_set_tri_staging(void *ctx, int32_t max_bytes) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (max_bytes < 0 || max_bytes > 220 * 1024) return fail(c, LT_ERR_ARG, "max_bytes must be in [0, 220 KiB]");
    c->smem_tri_bytes = max_bytes;
    batch_drop_graph(c);     // a captured batch step holds the old launch shape
    return LT_OK;
    LT_CATCH(ctx)
}

int lt_set_step_limit(void *ctx, int32_t max_steps) {
    LT_TRY
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (max_steps < 0) return fail(c, LT_ERR_ARG, "max_steps must be >= 0");
    c->max_steps = max_steps;
    batch_drop_graph(c);     // a captured batch step holds the old limit
    return LT_OK;
    LT_CATCH(ctx)
}

}  // extern "C"
