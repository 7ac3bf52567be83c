/* sg.h -- C ABI of the irradiance surrogate (libltrace.so).
 *
 * A learned model of the irradiance one unit-intensity spot light puts on
 * every texel of a scene, K(t, l), so that a lighting design's irradiance is
 * E_t = sum_l I_l K(t, l) with I_l = p_l^2 / 2 -- the linearity in emitted
 * power and the additivity over lights that the light tracer's texel
 * deposits have (Eq. 7-8). It is trained on the tracer's own irradiance and
 * serves as a cheap first stage of the design optimisation (Eq. 6 objective,
 * gradient with respect to the luminaire parameters as in Eq. 11); the
 * tracer stays both the fallback and the judge of the surrogate's error.
 *
 * Model: K = sigmoid(o_0) D + 0.01 softplus(o_1), where
 * D = a(theta) |cos_r| / r^2 is the unoccluded direct irradiance of the spot
 * (inverse-square cosine law, falloff a of Eq. S.11) and o = W3 relu(W2
 * relu(W1 relu(W0 x))) (no biases; W0..W2 64 x 64, W3 16 x 64) on the input
 *   x[0..31]  16-level hash encoding of the texel centre (Mueller et al.
 *             2022: 2 features per level, 2^19 entries per level, level
 *             resolutions 16, 20, 25, 32, 40, 50, 64, 80, 101, 128, 161, 203,
 *             256, 322, 406, 512 cells along the normalised box, dense
 *             indexing x + (N+1)(y + (N+1) z) for levels 0-6, spatial hash
 *             (x * 1 ^ y * 2654435761 ^ z * 805459861) mod 2^19 above),
 *             trilinear interpolation; the position is normalised in float32
 *             as (p - lo) * (1 / ext)
 *   x[32..34] u, unit vector from the texel centre to the light
 *   x[35]     r / 10            x[36..38] n_l, the spot axis
 *   x[39]     cos_l = -u . n_l  x[40] |n_t . u|      x[41] a(cos_l)
 *   x[42]     cos(theta_in)     x[43..45] (light position - lo) / ext
 *   x[46..48] n_t, texel normal x[49] 1              x[50..63] 0.
 * Weights are bf16 (an fp32 master copy is trained); every matrix product
 * takes bf16 inputs (x, hidden activations, back-propagated gradients) and
 * accumulates in fp32 on the tensor cores. The hash table is fp32.
 *
 * Training minimises (1 / B) sum_b 1/2 (A_t / mean A) (K_b - E_obs_b)^2 over
 * batches of (solve, texel) samples with Adam (beta 0.9 / 0.99, eps 1e-15,
 * bias-corrected), where solve s is a unit-intensity spot and E_obs[s] the
 * irradiance the tracer deposited for it.
 *
 * Conventions: every call returns an lt status (LT_OK = 0, negative on
 * error, message in sg_last_error); host inputs are copied; device pointers
 * are caller-owned and must stay valid for the calls that use them; all work
 * runs on the context's stream, and calls that return host values
 * synchronise it. No C++ exception crosses the interface (host memory
 * running out is LT_ERR_OOM). A context is not thread-safe: calls on one
 * context must not overlap; separate contexts share no state. The light
 * record is lt_light (lt.h); only spot lights are
 * modelled, and the surrogate gives no gradient for theta_out (it is trained
 * at one outer cone).
 */
#ifndef SG_H
#define SG_H

#include <stdint.h>

#include "lt.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SG_LEVELS 16
#define SG_TABLE_PER_LEVEL 524288                 /* 2^19 entries of 2 floats */
#define SG_TABLE_FLOATS (SG_LEVELS * SG_TABLE_PER_LEVEL * 2)
#define SG_WEIGHTS (3 * 64 * 64 + 16 * 64)        /* W0, W1, W2, W3 row-major [out][in] */
#define SG_IN 64
#define SG_OUT 16
#define SG_MAX_BATCH (1 << 20)

/* Create a surrogate context on CUDA device `device`, work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream). The context owns its
 * device buffers. LT_ERR_ARG for a NULL ctx_out; LT_ERR_CUDA when the device
 * does not exist or its buffers cannot be set up. */
LT_API int sg_create(void **ctx_out, int device, void *cuda_stream);

/* Free a context and its device memory after its stream drains; LT_ERR_ARG
 * for NULL. */
LT_API int sg_destroy(void *ctx);

/* Message of the context's last failed call, valid until the next call on
 * it; "null context" for NULL. */
LT_API const char *sg_last_error(const void *ctx);

/* Texel centres pos [n][3] and unit normals normal [n][3] (as lt_texel_centres
 * gives them), texel areas [n] (host, copied), and the normalised box: lo[3]
 * and the scalar extent ext > 0. Resets nothing else. */
LT_API int sg_set_texels(void *ctx, const float *pos, const float *normal, const float *area, int64_t n_texels,
                         const float *lo, float ext);

/* Parameters: weights [SG_WEIGHTS] fp32 (W0, W1, W2, W3, each row-major
 * [out][in]) and table [SG_TABLE_FLOATS] fp32 ([level][entry][feature]),
 * host or device (is_device). Setting resets the Adam moments and step. */
LT_API int sg_set_params(void *ctx, const float *weights, const float *table, int is_device);

/* Copy of the current parameters, laid out as for sg_set_params: the fp32
 * master weights and the table, into host or device memory (is_device).
 * LT_ERR_STATE before sg_set_params. */
LT_API int sg_get_params(void *ctx, float *weights, float *table, int is_device);

/* Training data: n_solves unit-intensity spots (host, copied) and their
 * observed texel irradiance E_obs [n_solves][n_texels] (device pointer,
 * caller-owned, read by every later sg_train_step). */
LT_API int sg_set_training_data(void *ctx, const lt_light *lights, int32_t n_solves, const float *E_obs);

/* One Adam step on a batch of `batch` samples (1..SG_MAX_BATCH). samples
 * [batch][2] = (solve, texel) pairs (host), or NULL to draw them on the
 * device with splitmix64 (Steele, Lea and Flood 2014) of `seed`, the step
 * number and the sample index. Writes the batch loss (before the update) to *loss_out (host,
 * may be NULL) and keeps the batch's gradients for sg_get_gradients. */
LT_API int sg_train_step(void *ctx, uint64_t seed, int32_t batch, float lr, const int32_t *samples,
                         double *loss_out);

/* Gradients of the last sg_train_step's loss (before its update) with
 * respect to the weights [SG_WEIGHTS] and the table [SG_TABLE_FLOATS]; host
 * or device. The table gradient is summed with float atomics, so its
 * rounding depends on the order in which the GPU ran them. */
LT_API int sg_get_gradients(void *ctx, float *dweights, float *dtable, int is_device);

/* K(t, light) of one light for every texel: K_out [n_texels], host or device. */
LT_API int sg_response(void *ctx, const lt_light *light, float *K_out, int is_device);

/* Design objective O = 1/2 sum_t A_t alpha_t (E_t - E*_t)^2 with
 * E_t = sum_l I_l K(t, l), and dO/dp [n_lights][LT_GRAD_N] in the order
 * (x, y, z, yaw, pitch, p_int, theta_in, theta_out = 0). lights: host
 * (copied); E_target, alpha: device [n_texels] (alpha may be NULL = 1);
 * loss_out and grad_out: host (either may be NULL); E_out: device
 * [n_texels] or NULL. */
LT_API int sg_design(void *ctx, const lt_light *lights, int32_t n_lights, const float *E_target, const float *alpha,
                     double *loss_out, double *grad_out, float *E_out);

/* The network alone on given input rows (test and inspection hook): X
 * [rows][SG_IN] host fp32 (rounded to bf16 like every input), O_out
 * [rows][SG_OUT]; if dO [rows][SG_OUT] is given, back-propagates it and
 * writes dX_out [rows][SG_IN] (may be NULL) and the weight gradient summed
 * over the rows, dW_out [SG_WEIGHTS] (may be NULL). All host. rows <=
 * SG_MAX_BATCH. */
LT_API int sg_network(void *ctx, const float *X, int32_t rows, const float *dO, float *O_out, float *dX_out,
                      float *dW_out);

/* Kernels of the network. flags: SG_KERNELS_DESIGN_TC runs the design
 * objective (sg_response and sg_design, forward and backward) on the
 * 5th-generation tensor cores (tcgen05.mma, fp32 accumulators in tensor
 * memory, four 128-row tiles per CTA), SG_KERNELS_TRAIN_TC does the same for
 * the training step's forward and backward (sg_train_step; two threads per
 * row, two 128-row tiles per CTA); a cleared flag
 * selects warp-level mma.sync (16 rows per warp) for that part. The default
 * is SG_KERNELS_DESIGN_TC alone, the measured faster pair: the training step
 * is bound by its hash-table gathers and atomics, where the two kernels are
 * within a few per cent and mma.sync leads. Both kernels of each part take
 * bf16 inputs
 * and accumulate in fp32; they agree up to the order of the fp32 sums (and,
 * in training, of the float atomics into the table gradient). Unknown flag
 * bits return LT_ERR_ARG. A tensor-core wait that gives up returns
 * LT_ERR_TIMEOUT (from sg_design, or from sg_train_step when it returns the
 * loss). */
#define SG_KERNELS_DESIGN_TC 1
#define SG_KERNELS_TRAIN_TC 2
LT_API int sg_set_kernels(void *ctx, int flags);

/* Hash encoding of normalised positions xn [rows][3] (host) with the
 * current table: enc_out [rows][32] (host). */
LT_API int sg_encode(void *ctx, const float *xn, int32_t rows, float *enc_out);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
