/*
 * lt.h -- C ABI of the GB300 light-tracing library (libltrace.so).
 *
 * View-independent adjoint light tracing (Lipp et al., "View-Independent
 * Adjoint Light Tracing for Lighting Design Optimization", arXiv 2310.02043):
 * a forward pass traces photons from parameterised luminaires and deposits
 * irradiance into per-texel storage on the scene surfaces; an L2 objective
 * compares it with a target; an adjoint pass replays the same photon paths
 * and accumulates the objective's gradient with respect to every luminaire
 * parameter.
 *
 * Conventions for every call:
 *   - Returns LT_OK (0) or a negative lt_status. A failed call leaves a
 *     message for lt_last_error(). No C++ exception crosses this interface:
 *     host memory running out is LT_ERR_OOM.
 *   - Fault injection for testing callers: with the environment variable
 *     LT_FAULT_HOST_ALLOC set and non-empty, the BVH build of lt_upload_scene
 *     and lt_build_bvh fails as if host memory ran out (LT_ERR_OOM); a context
 *     stays usable after it.
 *   - Work is queued on the context's CUDA stream (lt_create / lt_set_stream).
 *     Calls that return a value in host memory synchronise that stream.
 *   - Host input arrays are copied; the caller keeps ownership. Output
 *     pointers are caller-owned and must hold the stated number of elements.
 *   - A context is not thread-safe: calls on one context must not overlap
 *     (the caller serialises them). Separate contexts share no state, except
 *     the fixed scratch array of lt_loss_static (see there).
 *   - "is_device" arguments say whether a pointer is device memory (1) or
 *     host memory (0) of the context's device.
 *   - Light parameter / gradient slot order is LT_GRAD_*:
 *       [x, y, z, yaw, pitch, p_int, theta_in, theta_out].
 */
#ifndef LT_H
#define LT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LT_API __attribute__((visibility("default")))
#else
#define LT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LT_OK = 0,
    LT_ERR_ARG = -1,       /* invalid argument (sizes, ranges, null pointers) */
    LT_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    LT_ERR_OOM = -3,       /* device allocation failed */
    LT_ERR_STATE = -4,     /* call out of order (e.g. loss before a forward pass) */
    LT_ERR_TIMEOUT = -5,   /* a kernel gave up after its iteration limit */
    LT_ERR_OVERFLOW = -6,  /* fixed-point range exceeded */
    LT_ERR_DEVICE = -7     /* a kernel reported an internal error (device error word) */
} lt_status;

enum { LT_POINT = 0, LT_SPOT = 1, LT_AREA = 2 };

enum {
    LT_GRAD_X = 0, LT_GRAD_Y = 1, LT_GRAD_Z = 2, LT_GRAD_YAW = 3, LT_GRAD_PITCH = 4,
    LT_GRAD_P_INT = 5, LT_GRAD_THETA_IN = 6, LT_GRAD_THETA_OUT = 7, LT_GRAD_N = 8
};

/* One luminaire (Sec. 4.4 of the paper and the supplement's "Derivative
 * terms for optimization parameters"):
 *   type       LT_POINT, LT_SPOT or LT_AREA
 *   pos        position, metres (an area light's centroid)
 *   yaw,pitch  axis n = (cos p cos y, cos p sin y, sin p), z up (radians;
 *              the paper rotates by a rotation vector, Eq. 15)
 *   p_int      intensity parameter, I_e = p_int^2 / 2 (Sec. 4.4.1); for an
 *              area light the emitted power P = p_int^2 / 2
 *   theta_in   spot: inner cone half-angle, full intensity for theta <= theta_in;
 *              area: width (metres) along t = dn/dpitch
 *   theta_out  spot: outer cone half-angle, zero beyond; quadratic soft edge in
 *              cos(theta) between the two (Eq. S.11), 0 <= theta_in < theta_out <= pi;
 *              area: height (metres) along b = n x t
 * Point lights ignore yaw, pitch and the cone angles. An area light is a
 * Lambertian rectangle (supplement, Eq. S.15-S.16): rays start uniformly on
 * it and leave uniformly over the hemisphere about n with flux
 * Phi_r = 2 P cos(theta) / N; its gradient slots 6 and 7 stay 0. */
typedef struct {
    int32_t type;
    float pos[3];
    float yaw;
    float pitch;
    float p_int;
    float theta_in;
    float theta_out;
} lt_light;

/* Counters of the last passes and facts about the uploaded scene. */
typedef struct {
    uint64_t segments_forward;   /* traced segments (hit or miss) of the last forward pass */
    uint64_t segments_adjoint;   /* same for the last adjoint pass */
    uint64_t photons_forward;
    uint64_t photons_adjoint;
    int64_t n_texels;
    int32_t n_triangles;
    int32_t n_nodes;             /* wide-BVH nodes */
    int32_t bvh_depth;           /* levels of wide nodes */
    int32_t staged_nodes;        /* nodes held in shared memory per block */
    double fixed_point_scale;    /* S of the last forward pass (single or batch): a texel accumulates round(Phi * S) */
    int32_t grid_blocks;         /* launch shape of the last forward pass (single or batch) */
    int32_t block_threads;
    int32_t staged_triangles;    /* triangles held in shared memory per block (last forward pass) */
    int32_t reserved;
} lt_stats;

/* Library ABI version (this header: 2). */
LT_API int lt_version(void);

/* Create a context on CUDA device `device`; work goes to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). The context owns every
 * device buffer it allocates. LT_ERR_ARG for a NULL ctx_out or a device
 * index out of range, LT_ERR_CUDA if the device cannot be set up; *ctx_out
 * is NULL on failure. */
LT_API int lt_create(void **ctx_out, int device, void *cuda_stream);

/* Free a context and all its device and pinned host memory (waits for its
 * stream). NULL is allowed and does nothing. */
LT_API int lt_destroy(void *ctx);

/* Queue later work of the context on `cuda_stream` (a cudaStream_t of the
 * context's device; the caller keeps it alive). Work already queued is not
 * moved: order the two streams if they overlap. */
LT_API int lt_set_stream(void *ctx, void *cuda_stream);

/* Message of the context's last failed call ("" if none), valid until the
 * next call on the context; "null context" for NULL. */
LT_API const char *lt_last_error(const void *ctx);

/* Upload a triangle scene (host arrays, copied) and build its wide BVH.
 *   tri_xyz    [n_tri][3][3] float   vertex positions
 *   tri_uv     [n_tri][3][2] float   per-vertex chart coordinates in [0,1]^2
 *   tri_tile   [n_tri] int32         tile (texel chart) of each triangle
 *   tri_albedo [n_tri] float         Lambertian albedo in [0, 1]
 *   tile_res   [n_tiles][2] int32    texel resolution (res_u, res_v) >= 1
 *   tile_area  [n_tiles] double      area covered by the tile, m^2 (> 0)
 * Texels are numbered tile by tile, u fastest. A texel's area is
 * tile_area / (res_u res_v) (the box basis standing in for the per-vertex
 * hat basis of Eq. 4; mass-lumped projection, Eq. S.6). Writes the texel
 * count to *n_texels_out. Invalidates targets, weights and pass results.
 * The BVH is kept as float nodes (staged in shared memory when it fits) and
 * as compressed nodes (lt_compress_bvh, read through L1 otherwise); a scene
 * whose BVH has a node wider than about 2e6 along an axis is refused
 * (LT_ERR_ARG). An argument error or a failed BVH build leaves the previous
 * scene in place. */
LT_API int lt_upload_scene(void *ctx, const float *tri_xyz, const float *tri_uv, const int32_t *tri_tile,
                    const float *tri_albedo, int32_t n_tri, const int32_t *tile_res, const double *tile_area,
                    int32_t n_tiles, int64_t *n_texels_out);

/* One node of the 8-wide BVH (240 bytes), the layout the traversal kernels
 * read from device memory. Slot k (0..7) holds a child with the box
 * [lo_x[k], hi_x[k]] x [lo_y[k], hi_y[k]] x [lo_z[k], hi_z[k]]: the float
 * bounds of its triangles grown by a margin on every side, so that a plane
 * distance rounded by the traversal never cuts a triangle off. child[k] >= 0
 * is an inner node (bit k of inner_mask set); INT32_MIN is an empty slot,
 * whose box is inverted (lo > hi) so that no ray enters it; any other
 * negative value is a leaf of ((-1 - child[k]) & 3) + 1 triangles starting
 * at leaf-order position (-1 - child[k]) >> 2. Slot k faces the direction
 * whose component a is + when bit a of k is set: children are assigned to
 * slots so that the sum over children of -dot(child centre - node centre,
 * slot direction) is least, which lets the traversal visit near children
 * first by a per-ray XOR of the slot index. */
typedef struct {
    float lo_x[8], hi_x[8], lo_y[8], hi_y[8], lo_z[8], hi_z[8];
    int32_t child[8];
    uint32_t inner_mask;
    uint32_t pad[3];
} lt_bvh_node;

/* Build the wide BVH of n_tri triangles (tri_xyz as for lt_upload_scene) on
 * the host, without a context or a device: the same builder lt_upload_scene
 * runs, exposed for inspection. Nodes are breadth-first (node 0 is the root,
 * parents come before their children). Outputs, each optional (NULL):
 *   nodes_out    [nodes_cap] lt_bvh_node
 *   order_out    [n_tri] int32: leaf-order position -> input triangle index
 *   n_nodes_out  node count; depth_out levels of wide nodes (<= 16)
 * Returns LT_ERR_ARG for an empty or non-finite input, for a tree deeper
 * than 16 levels, or when nodes_cap is below the node count (the counts are
 * still written); LT_ERR_OOM when host memory runs out. */
LT_API int lt_build_bvh(const float *tri_xyz, int32_t n_tri, lt_bvh_node *nodes_out, int32_t nodes_cap,
                        int32_t *order_out, int32_t *n_nodes_out, int32_t *depth_out);

/* Compressed 8-wide node (96 bytes), the form the tracing kernels read when
 * the BVH is not staged in shared memory (quantised child boxes). Per axis a
 * (x, y, z): a float origin origin[a] and a step 2^e_a, where byte a of meta
 * holds e_a + 142; child k's box along a is
 * [origin[a] + q[a][k] 2^e_a, origin[a] + q[a][8 + k] 2^e_a]. Every box
 * contains the float node's box widened by 2^-14 of the node's extent
 * along a (the rounding of the kernel's decode); empty slots hold
 * q lo = 255, q hi = 0. Byte 3 of meta is the inner mask; child[] is the
 * float node's. */
typedef struct {
    float origin[3];
    uint32_t meta;
    uint8_t q[3][16];
    int32_t child[8];
} lt_bvh_cnode;

/* Compress n_nodes nodes of lt_build_bvh into out[n_nodes] (host only, the
 * conversion lt_upload_scene runs). LT_ERR_ARG for null pointers, a
 * non-positive count, a non-empty slot with a non-finite or inverted box, or
 * a node wider than about 2e6 along an axis (the range of the kernels'
 * decode; lt_upload_scene refuses such a scene the same way). */
LT_API int lt_compress_bvh(const lt_bvh_node *nodes, int32_t n_nodes, lt_bvh_cnode *out);

/* Target irradiance E*_t and weights alpha_t of the objective (Eq. 6),
 * [n_texels] floats each; alpha may be NULL (all ones). */
LT_API int lt_set_target(void *ctx, const float *E_target, const float *alpha, int is_device);

/* Luminaires, host array of n_lights (1..LT_MAX_LIGHTS), copied. */
#define LT_MAX_LIGHTS 1024
LT_API int lt_set_lights(void *ctx, const lt_light *lights, int32_t n_lights);

/* Forward pass (Alg. 1): photons [photon_begin, photon_end) of a budget of
 * n_photons split evenly over the lights (light l owns a contiguous range;
 * the first n_photons mod n_lights lights take one extra photon). Each photon
 * is traced for up to max_hits surface hits (1..64): it deposits its flux
 * Phi_i at every hit (Eq. 8, order 0) and continues in a cosine-weighted
 * direction with Phi_{i+1} = rho Phi_i (Eq. 7). Random numbers are
 * Philox4x32-10 with counter (photon lo, photon hi, segment, 0) and key
 * (seed lo, seed hi). Clears and then fills the texel accumulator, a
 * [n_texels] int64 fixed-point array (value round(Phi * S)); the result is
 * bit-reproducible for any launch configuration. A pass covers at most
 * 2^32 - 1 photons (photon_end - photon_begin; larger ranges are
 * LT_ERR_ARG: split them, the integer sums add up exactly); the same holds
 * for lt_trace_adjoint, lt_count_work and lt_debug_paths. */
LT_API int lt_trace_forward(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                     uint64_t photon_end);

/* Device pointer of the int64 texel accumulator and its scale S (valid until
 * the next lt_upload_scene). Ranks that split photons can sum these arrays
 * (exact integer addition) before lt_loss. */
LT_API int lt_texel_accumulator(void *ctx, int64_t **q_device, double *scale_out);

/* Copy of the int64 texel accumulator ([n_texels]) into caller memory. */
LT_API int lt_get_texel_sums(void *ctx, int64_t *q_out, int is_device);

/* Objective (Eq. 6, order 0): O = 1/2 sum_t A_t alpha_t (E_t - E*_t)^2 with
 * E_t = q_t / (S A_t). Also forms the adjoint weights
 * w_t = alpha_t (E_t - E*_t) = dO/dPhi for a deposit into texel t, kept on the
 * device for lt_trace_adjoint. Writes O (double) to loss_out. Deterministic. */
LT_API int lt_loss(void *ctx, double *loss_out, int is_device);

/* Irradiance E_t (float, [n_texels]) of the last forward pass. */
LT_API int lt_get_irradiance(void *ctx, float *E_out, int is_device);

/* Texel areas A_t (float, [n_texels]). */
LT_API int lt_texel_areas(void *ctx, float *A_out, int is_device);

/* Centre of every texel in world space and the unit normal of its tile
 * (host arrays [n_texels][3]): the point whose chart coordinates are
 * ((i + 1/2) / res_u, (j + 1/2) / res_v) in texel (i, j) of its tile, mapped
 * through the barycentric coordinates of the tile triangle that contains it
 * in the chart (the one whose smallest barycentric coordinate is largest,
 * clamped onto that triangle if none contains it). Inputs of the irradiance
 * surrogate (sg.h); computed on the host from the uploaded scene. */
LT_API int lt_texel_centres(void *ctx, float *pos_out, float *normal_out);

/* Replace the adjoint weights w_t ([n_texels] floats) -- injects dO/dPhi
 * directly (for gradient checks against closed forms). */
LT_API int lt_set_adjoint_weights(void *ctx, const float *w, int is_device);

/* Adjoint pass (Alg. 2, Eq. 11-12): replays photons [photon_begin,
 * photon_end) of the budget n_photons from `seed` (the forward seed for a
 * correlated estimate, another for a decorrelated one, Sec. 4.3). Per photon
 * the adjoint state dO/dPhi_r = sum_i w_{t_i} prod_{j<i} rho_j is summed along
 * the path and multiplied by dPhi_r/dp, taken at the first hit with that hit
 * held fixed (Sec. 4.4.2: Eq. 14 for position, Eq. S.11-S.12 for the spot
 * edge, Eq. 15 for orientation, I_e = p^2/2 for intensity). Writes dO/dp as
 * double [n_lights][LT_GRAD_N] to grad_out. Needs weights from lt_loss or
 * lt_set_adjoint_weights. Exact summation: every photon's term (a float) is
 * multiplied by the gradient scale G = 2^-e, e the binary exponent of
 * max_t |w_t| times the largest flux constant I_e Omega / N_l of the lights
 * (the size of a typical term), rounded to a multiple of 2^-64 and added as
 * a 128-bit two's-complement integer; the integer sums are converted once,
 * correctly rounded, to double and scaled by 2^-64 / G. The result is
 * therefore bitwise the same for every launch shape, and the integer sums
 * of a partition of the photon range add up exactly to those of the whole
 * (lt_gradient_fixed). A term that is not finite or reaches 2^62 / G
 * returns LT_ERR_OVERFLOW. The pass keeps a 16-byte record per photon of
 * the range (its adjoint state and first hit) between its trace kernel and
 * its gradient kernel; the context holds that buffer and reuses it. */
LT_API int lt_trace_adjoint(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                     uint64_t photon_end, double *grad_out, int is_device);

/* The exact gradient sums of the last lt_trace_adjoint: per light and slot
 * ([n_lights][LT_GRAD_N]) a 128-bit two's-complement integer as two int64,
 * low word first (sums_out: [n_lights][LT_GRAD_N][2] host), and the scale G
 * (scale_out, host): dO/dp = integer x 2^-64 / G. Callers that split the
 * photons of one budget over several passes or ranks (same weights, same
 * lights, so the same G) add these integers (exactly, e.g. in 128-bit or
 * arbitrary-precision arithmetic) and convert the sum once; the result
 * equals the gradient of one pass over the whole range bit for bit.
 * Synchronises the context's stream. LT_ERR_STATE before any adjoint pass. */
LT_API int lt_gradient_fixed(void *ctx, int64_t *sums_out, double *scale_out);

/* Debug record of photons [photon_begin, photon_begin + count): original
 * triangle index and texel of every hit, -1 after the path ends (host
 * outputs [count][max_hits]). If grad_out is not NULL it receives every
 * photon's own gradient term dO/dPhi_r * dPhi_r/dp (host [count][LT_GRAD_N],
 * double; needs adjoint weights as lt_trace_adjoint does). */
LT_API int lt_debug_paths(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                   uint64_t count, int32_t *tri_out, int64_t *texel_out, double *grad_out);

/* Counters of the last forward and adjoint passes and facts about the
 * uploaded scene (lt_stats above), copied into caller memory. Synchronises
 * the context's stream (the segment counters are read from the device). */
LT_API int lt_get_stats(void *ctx, lt_stats *out);

/* Forward pass exactly as lt_trace_forward (same texel sums) through a
 * counting variant of the kernel, for work accounting: writes
 * counts_out[0] = segments traced, [1] = BVH node visits, [2] =
 * ray/triangle tests, [3] = photons. */
LT_API int lt_count_work(void *ctx, uint64_t seed, uint64_t n_photons, int32_t max_hits, uint64_t photon_begin,
                  uint64_t photon_end, uint64_t *counts_out);

/* Philox design word (counter word 3) of the single-design passes; default
 * 0. A design traced in a batch (lt_batch_*) as design d follows the same
 * photon paths as a single-design pass with design word d; its irradiance,
 * objective and gradient agree with that pass up to the rounding of the
 * fixed-point scale (a batch sizes one power-of-two scale for its brightest
 * design). */
LT_API int lt_set_design(void *ctx, uint32_t design);

/* ---- Batched designs -----------------------------------------------------
 * Many candidate lighting designs of one scene, with uneven light counts,
 * traced in one launch per pass: design d owns photons [d N, (d + 1) N) of
 * the launch (N photons per design, split evenly over its lights) and its
 * own texel sums, irradiance, weights and objective against the shared
 * target (lt_set_target). The Philox design word of design d is d. A step
 * uploads the lights and seeds, runs the forward pass, the per-design
 * objective and the adjoint pass, and returns the objectives and gradients.
 * It can run as a captured CUDA graph, instantiated on the first such step
 * and replayed afterwards (seeds and the fixed-point scale are read from
 * device memory the graph refreshes, so one graph serves every step; it is
 * rebuilt after lt_set_launch or lt_batch_setup). Batch work runs on the
 * context's own non-blocking stream and every step synchronises it; do not
 * overlap batch steps with single-design passes of the same context. */
#define LT_MAX_BATCH_LIGHTS 65536

/* Allocate a batch: n_designs designs with lights_per_design[d] >= 1 lights
 * each (at most LT_MAX_BATCH_LIGHTS in total), photons_per_design photons and
 * max_hits hits per photon; n_designs x photons_per_design at most
 * 2^32 - 1 (LT_ERR_ARG otherwise). Needs an uploaded scene; replaces a
 * previous batch. Device memory: n_designs x n_texels x 16 bytes plus small
 * buffers. */
LT_API int lt_batch_setup(void *ctx, int32_t n_designs, const int32_t *lights_per_design,
                          uint64_t photons_per_design, int32_t max_hits);

/* Lights of every design, concatenated in design order (host, copied). */
LT_API int lt_batch_set_lights(void *ctx, const lt_light *lights);

/* One step: forward (seed_fwd), objective, adjoint (seed_adj). Writes the
 * objective of every design to loss_out [n_designs] and dO/dp of every light
 * to grad_out [total lights][LT_GRAD_N] (host, either may be NULL).
 * use_graph = 1 replays a captured CUDA graph of the step. */
LT_API int lt_batch_step(void *ctx, uint64_t seed_fwd, uint64_t seed_adj, double *loss_out, double *grad_out,
                         int use_graph);

/* The context's batch stream (a cudaStream_t), valid from lt_batch_setup
 * until the next lt_batch_setup or lt_destroy; NULL before the first setup.
 * Callers order their own work after a step, or record CUDA events around
 * one, on this stream. */
LT_API int lt_batch_stream(void *ctx, void **stream_out);

/* Texel sums (int64 [n_texels], fixed point with the batch's scale) of one
 * design after a step, into host or device memory (is_device). */
LT_API int lt_batch_texel_sums(void *ctx, int32_t design, int64_t *q_out, int is_device);

/* Irradiance (float [n_texels]) of one design after a step, into host or
 * device memory (is_device). */
LT_API int lt_batch_irradiance(void *ctx, int32_t design, float *E_out, int is_device);

/* Objective and adjoint weights for callers that cannot allocate device
 * memory. The paper has no counterpart: this is a deployment variant of
 * lt_loss.
 *
 * Some callers must not call cudaMalloc: code running inside a memory pool
 * that another framework owns (its allocator would not see the block), or a
 * device already at its memory budget.
 * This call allocates nothing. The caller passes every input and output as
 * device pointers on `device`; the only scratch, one double per block of
 * 4096 texels, lives in a fixed 32 KiB array compiled into the library, which
 * every device that loads the library holds until the process exits.
 *   q         [n_texels] int64 fixed-point texel sums (lt_texel_accumulator)
 *   scale     their scale S > 0: E_t = q_t / (S A_t)
 *   area      [n_texels] texel areas A_t (lt_texel_areas)
 *   E_target  [n_texels] target E*_t; alpha [n_texels] weights, or NULL (ones)
 *   w_out     [n_texels] adjoint weights alpha_t (E_t - E*_t)
 *   E_out     [n_texels] irradiance E_t, or NULL
 *   loss_out  one device double: O = 1/2 sum_t A_t alpha_t (E_t - E*_t)^2
 * n_texels must lie in [1, LT_LOSS_STATIC_MAX_TEXELS]; larger inputs return
 * LT_ERR_ARG (use lt_loss). Work is queued on cuda_stream, nothing is
 * synchronised; the calling thread's current device is restored. The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress). The address is kept for the life of the process: after cudaDeviceReset
 * (or anything else that replaces the device's primary context) this call
 * must not be used on that device again. If a CUDA error from earlier work
 * is pending on the calling thread, the call returns LT_ERR_STATE without
 * launching and leaves that error pending.
 * All calls on a device share the array -- nothing in it needs clearing, each
 * call writes every slot it reads -- so calls that overlap on the GPU (two
 * streams, two threads) race: order them on one stream. Returns only a
 * status (there is no context for lt_last_error). O equals lt_loss's up to
 * the order of the floating-point sum; w_out and E_out are the same values. */
#define LT_LOSS_STATIC_MAX_TEXELS 16777216
LT_API int lt_loss_static(int device, void *cuda_stream, const int64_t *q, double scale, const float *area,
                          const float *E_target, const float *alpha, int64_t n_texels, float *w_out,
                          float *E_out, double *loss_out);

/* Launch shape of the tracing kernels. threads_per_block: a multiple of 32
 * up to 1024, 0 = the bound of the kernel the BVH selects (1024, both for
 * the kernels that stage the BVH in shared memory and for those that read
 * nodes through L1; the bounds are build-time constants); a trace whose BVH
 * selects a kernel with a smaller bound than the request fails with
 * LT_ERR_ARG. blocks_per_sm: resident blocks per SM, 0 = as many
 * as fit. smem_node_bytes: shared-memory budget for staged BVH nodes in
 * [0, 200 KiB] (the whole BVH is staged when it fits, else none), 0 = stage
 * nothing. A negative argument keeps the current value. The defaults are the
 * kernel's bound, as many blocks as fit, 72 KiB. */
LT_API int lt_set_launch(void *ctx, int32_t threads_per_block, int32_t blocks_per_sm, int32_t smem_node_bytes);

/* Shared-memory budget for staging the triangles with the nodes: when the
 * whole BVH is staged (lt_set_launch) and the nodes, their parent links and
 * all triangles (52 bytes each there) take at most max_bytes, and the extra
 * shared memory leaves as many blocks resident per SM as without it (the
 * requested blocks_per_sm, else as many as fit), every block copies the
 * triangles to shared memory too, and the leaf tests read them there.
 * max_bytes in [0, 220 KiB]; 0 = never; default 200 KiB. Results do not
 * depend on it (the same tests on the same values). Takes effect at the next
 * trace; a captured batch graph is rebuilt. */
LT_API int lt_set_tri_staging(void *ctx, int32_t max_bytes);

/* Give-up limit of the tracing kernels: BVH node visits one ray may make
 * before the kernel ends that ray as a miss, records the give-up in the
 * device error word and carries on (no kernel waits or traps). The next call
 * that synchronises (lt_get_stats, lt_loss or lt_trace_adjoint into host
 * memory, ...) then returns LT_ERR_TIMEOUT once and clears the word; the
 * context stays usable. max_steps >= 1 sets the limit, 0 restores the
 * default (16 x BVH nodes + 64, more than any ray of a valid tree needs);
 * negative is LT_ERR_ARG. A test hook for that error path. */
LT_API int lt_set_step_limit(void *ctx, int32_t max_steps);

/* L2 read bandwidth of `device` (no context; a measurement aid, not part of
 * the paper's method): a buffer of `bytes` (1 MiB .. 96 MiB, so it stays
 * in the 129 MB L2) is swept `reps` times with 16-byte loads cached in L2
 * only, after one warm-up sweep; writes the best of five timed runs (CUDA
 * events) in GB/s to *gbs_out. Allocates and frees its own buffer and
 * stream, synchronises, restores the calling thread's current device.
 * LT_ERR_ARG for sizes out of range, LT_ERR_OOM / LT_ERR_CUDA on failure. */
LT_API int lt_probe_l2_read(int device, uint64_t bytes, int32_t reps, double *gbs_out);

#ifdef __cplusplus
}
#endif

#endif /* LT_H */
