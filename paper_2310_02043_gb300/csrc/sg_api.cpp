// sg_api.cpp -- C ABI of the irradiance surrogate (include/sg.h): device
// buffers, argument checks, and the order of the kernel launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/sg.h"
#include "sg_internal.h"

using namespace sg;

namespace {

struct SgCtx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // texels
    int64_t n = 0, n_pad = 0;
    float lo[3] = {0, 0, 0}, ext = 1.0f, inv_ext = 1.0f, inv_mean_area = 1.0f;
    float4 *d_pos = nullptr, *d_nrm = nullptr;
    float *d_area = nullptr;
    // parameters (fp32 master, bf16 copy), Adam moments, gradients
    float *d_W = nullptr, *d_mW = nullptr, *d_vW = nullptr, *d_gW = nullptr;
    uint16_t *d_Wb = nullptr;
    float *d_table = nullptr, *d_mT = nullptr, *d_vT = nullptr, *d_gT = nullptr;
    bool has_params = false;
    int64_t step = 0;
    uint16_t *d_enc = nullptr;
    bool enc_dirty = true;
    // training data
    LightC *d_train = nullptr;
    int32_t n_solves = 0;
    const float *E_obs = nullptr;
    // row buffers (train steps and sg_network)
    RowBuffers rb{nullptr, nullptr, 0};
    float *d_wpart = nullptr;
    size_t wpart_floats = 0;
    double *d_lpart = nullptr, *d_loss = nullptr;
    int32_t *d_samples = nullptr;
    int32_t samples_cap = 0;
    float *d_X = nullptr, *d_dO = nullptr, *d_O = nullptr, *d_dX = nullptr, *d_xn = nullptr, *d_enc_out = nullptr;
    size_t scratch_floats = 0;
    // design
    LightC *d_dl = nullptr;
    int32_t dl_cap = 0;
    float *d_K = nullptr, *d_up = nullptr, *d_gpart = nullptr;
    size_t K_floats = 0, up_floats = 0, gpart_floats = 0;
    double *d_dout = nullptr;
    int32_t *d_err = nullptr;                 // device error word of the tcgen05 kernels
    int use_tc = 1;                           // design objective on tcgen05 (1) or mma.sync (0)
    int train_tc = 0;                         // training network on tcgen05 (1) or mma.sync (0)
    double *h_pinned = nullptr;
    size_t h_pinned_bytes = 0;
};

int fail(SgCtx *c, int code, const std::string &msg) {
    c->err = msg;
    return code;
}

int cuda_fail(SgCtx *c, cudaError_t e, const char *what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA;
}

// No C++ exception crosses the C ABI: every entry point runs its body between
// LT_TRY and LT_CATCH, which turn an exception into a status and, when there
// is a context, its message. Called only from inside a catch handler.
int exception_status(SgCtx *c) noexcept {
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

#define LT_TRY try {
#define LT_CATCH(ctx)                                        \
    }                                                        \
    catch (...) {                                            \
        return exception_status(static_cast<SgCtx *>(ctx));  \
    }

#define SG_CUDA(c, expr)                                   \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
    } while (0)

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

template <typename T>
cudaError_t dalloc(T *&p, size_t count) {
    dfree(p);
    return cudaMalloc((void **)&p, count * sizeof(T) + 16);
}

// Grows a device buffer to hold at least `count` elements.
template <typename T>
cudaError_t ensure(T *&p, size_t &cap, size_t count) {
    if (p && cap >= count) return cudaSuccess;
    cudaError_t e = dalloc(p, count);
    cap = e == cudaSuccess ? count : 0;
    return e;
}

TexelView view(const SgCtx *c) {
    TexelView t;
    t.pos = c->d_pos;
    t.nrm = c->d_nrm;
    t.area = c->d_area;
    t.n = c->n;
    t.n_pad = c->n_pad;
    for (int a = 0; a < 3; ++a) t.lo[a] = c->lo[a];
    t.inv_ext = c->inv_ext;
    t.ext = c->ext;
    t.inv_mean_area = c->inv_mean_area;
    return t;
}

// Spot constants in double, rounded to float.
int derive(SgCtx *c, const lt_light *in, int32_t n, std::vector<LightC> *out) {
    out->resize((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const lt_light &L = in[i];
        if (L.type != LT_SPOT) return fail(c, LT_ERR_ARG, "the surrogate models spot lights only");
        if (!(L.theta_in >= 0.0f && L.theta_in < L.theta_out && L.theta_out < 3.14159265f))
            return fail(c, LT_ERR_ARG, "spot cones must satisfy 0 <= theta_in < theta_out < pi");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(L.pos[a])) return fail(c, LT_ERR_ARG, "non-finite light position");
        LightC &o = (*out)[(size_t)i];
        std::memset(&o, 0, sizeof(o));
        const double y = L.yaw, p = L.pitch, cy = std::cos(y), sy = std::sin(y), cp = std::cos(p), sp = std::sin(p);
        for (int a = 0; a < 3; ++a) o.p[a] = L.pos[a];
        o.nl[0] = (float)(cp * cy);
        o.nl[1] = (float)(cp * sy);
        o.nl[2] = (float)sp;
        o.dny[0] = (float)(-cp * sy);
        o.dny[1] = (float)(cp * cy);
        o.dny[2] = 0.0f;
        o.dnp[0] = (float)(-sp * cy);
        o.dnp[1] = (float)(-sp * sy);
        o.dnp[2] = (float)cp;
        const double ci = std::cos((double)L.theta_in), co = std::cos((double)L.theta_out);
        o.ci = (float)ci;
        o.co = (float)co;
        o.inv_dc = (float)(1.0 / (ci - co));
        o.sin_in = (float)std::sin((double)L.theta_in);
        o.p_int = L.p_int;
        o.intensity = (float)(0.5 * (double)L.p_int * (double)L.p_int);
    }
    return LT_OK;
}

int need_params(SgCtx *c) {
    if (!c->n) return fail(c, LT_ERR_STATE, "no texels (sg_set_texels)");
    if (!c->has_params) return fail(c, LT_ERR_STATE, "no parameters (sg_set_params)");
    return LT_OK;
}

int ensure_rows(SgCtx *c, int32_t rows) {
    const int32_t cap = (rows + 15) / 16 * 16;
    if (c->rb.rows < cap) {
        dfree(c->rb.act);
        dfree(c->rb.dz);
        c->rb.rows = 0;
        SG_CUDA(c, cudaMalloc((void **)&c->rb.act, (size_t)4 * cap * 64 * sizeof(uint16_t)));
        SG_CUDA(c, cudaMalloc((void **)&c->rb.dz, ((size_t)3 * cap * 64 + (size_t)cap * 16) * sizeof(uint16_t)));
        c->rb.rows = cap;
    }
    const size_t chunks = (size_t)(rows + kWgradChunk - 1) / kWgradChunk;
    SG_CUDA(c, ensure(c->d_wpart, c->wpart_floats, chunks * kWgradItems * 1024));
    return LT_OK;
}

int ensure_pinned(SgCtx *c, size_t bytes) {
    if (c->h_pinned_bytes >= bytes) return LT_OK;
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    c->h_pinned = nullptr;
    c->h_pinned_bytes = 0;
    SG_CUDA(c, cudaMallocHost((void **)&c->h_pinned, bytes));
    c->h_pinned_bytes = bytes;
    return LT_OK;
}

int refresh_encoding(SgCtx *c) {
    if (!c->enc_dirty) return LT_OK;
    SG_CUDA(c, launch_encode_texels(view(c), c->d_table, c->d_enc, c->stream));
    c->enc_dirty = false;
    return LT_OK;
}

void free_all(SgCtx *c) {
    dfree(c->d_pos); dfree(c->d_nrm); dfree(c->d_area);
    dfree(c->d_W); dfree(c->d_mW); dfree(c->d_vW); dfree(c->d_gW); dfree(c->d_Wb);
    dfree(c->d_table); dfree(c->d_mT); dfree(c->d_vT); dfree(c->d_gT); dfree(c->d_enc);
    dfree(c->d_train); dfree(c->rb.act); dfree(c->rb.dz); dfree(c->d_wpart);
    dfree(c->d_lpart); dfree(c->d_loss); dfree(c->d_samples);
    dfree(c->d_X); dfree(c->d_dO); dfree(c->d_O); dfree(c->d_dX); dfree(c->d_xn); dfree(c->d_enc_out);
    dfree(c->d_dl); dfree(c->d_K); dfree(c->d_up); dfree(c->d_gpart); dfree(c->d_dout); dfree(c->d_err);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    c->h_pinned = nullptr;
}

int copy_to(SgCtx *c, void *dst, const void *src, size_t bytes, int dst_is_device) {
    SG_CUDA(c, cudaMemcpyAsync(dst, src, bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               c->stream));
    if (!dst_is_device) SG_CUDA(c, cudaStreamSynchronize(c->stream));
    return LT_OK;
}

}  // namespace

extern "C" {

int sg_create(void **ctx_out, int device, void *cuda_stream) {
    LT_TRY
    if (!ctx_out) return LT_ERR_ARG;
    *ctx_out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return LT_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return LT_ERR_CUDA;
    SgCtx *c = new SgCtx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaMalloc((void **)&c->d_W, kWeights * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_mW, kWeights * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_vW, kWeights * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_gW, kWeights * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_Wb, kWeights * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_table, kTableFloats * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_mT, kTableFloats * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_vT, kTableFloats * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_gT, kTableFloats * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_lpart, 4096 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_loss, 16 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int32_t)) != cudaSuccess) {
        free_all(c);
        delete c;
        return LT_ERR_OOM;
    }
    *ctx_out = c;
    return LT_OK;
    LT_CATCH(nullptr)
}

int sg_destroy(void *ctx) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c) return LT_ERR_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return LT_OK;
    LT_CATCH(ctx)
}

const char *sg_last_error(const void *ctx) {
    const SgCtx *c = static_cast<const SgCtx *>(ctx);
    return c ? c->err.c_str() : "null context";
}

int sg_set_texels(void *ctx, const float *pos, const float *normal, const float *area, int64_t n_texels,
                  const float *lo, float ext) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c) return LT_ERR_ARG;
    if (!pos || !normal || !area || !lo || n_texels <= 0) return fail(c, LT_ERR_ARG, "null texel array or no texels");
    if (!(ext > 0.0f) || !std::isfinite(ext)) return fail(c, LT_ERR_ARG, "ext must be finite and > 0");
    SG_CUDA(c, cudaSetDevice(c->device));
    const int64_t n_pad = (n_texels + 15) / 16 * 16;
    std::vector<float4> P((size_t)n_pad), N((size_t)n_pad);
    std::vector<float> A((size_t)n_pad, 0.0f);
    double sum_a = 0.0;
    for (int64_t t = 0; t < n_pad; ++t) {
        if (t < n_texels) {
            P[(size_t)t] = make_float4(pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], 0.0f);
            N[(size_t)t] = make_float4(normal[3 * t], normal[3 * t + 1], normal[3 * t + 2], 0.0f);
            if (!(area[t] >= 0.0f) || !std::isfinite(area[t])) return fail(c, LT_ERR_ARG, "texel areas must be >= 0");
            A[(size_t)t] = area[t];
            sum_a += area[t];
        } else {
            P[(size_t)t] = make_float4(lo[0], lo[1], lo[2], 0.0f);
            N[(size_t)t] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
        }
    }
    if (!(sum_a > 0.0)) return fail(c, LT_ERR_ARG, "total texel area must be > 0");
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    SG_CUDA(c, dalloc(c->d_pos, (size_t)n_pad));
    SG_CUDA(c, dalloc(c->d_nrm, (size_t)n_pad));
    SG_CUDA(c, dalloc(c->d_area, (size_t)n_pad));
    SG_CUDA(c, dalloc(c->d_enc, (size_t)n_pad * 32));
    SG_CUDA(c, cudaMemcpy(c->d_pos, P.data(), P.size() * sizeof(float4), cudaMemcpyHostToDevice));
    SG_CUDA(c, cudaMemcpy(c->d_nrm, N.data(), N.size() * sizeof(float4), cudaMemcpyHostToDevice));
    SG_CUDA(c, cudaMemcpy(c->d_area, A.data(), A.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->n = n_texels;
    c->n_pad = n_pad;
    for (int a = 0; a < 3; ++a) c->lo[a] = lo[a];
    c->ext = ext;
    c->inv_ext = (float)(1.0 / (double)ext);
    c->inv_mean_area = (float)((double)n_texels / sum_a);
    c->enc_dirty = true;
    c->n_solves = 0;
    c->E_obs = nullptr;
    return LT_OK;
    LT_CATCH(ctx)
}

int sg_set_params(void *ctx, const float *weights, const float *table, int is_device) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !weights || !table) return LT_ERR_ARG;
    SG_CUDA(c, cudaSetDevice(c->device));
    const cudaMemcpyKind k = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SG_CUDA(c, cudaMemcpyAsync(c->d_W, weights, kWeights * sizeof(float), k, c->stream));
    SG_CUDA(c, cudaMemcpyAsync(c->d_table, table, kTableFloats * sizeof(float), k, c->stream));
    SG_CUDA(c, cudaMemsetAsync(c->d_mW, 0, kWeights * sizeof(float), c->stream));
    SG_CUDA(c, cudaMemsetAsync(c->d_vW, 0, kWeights * sizeof(float), c->stream));
    SG_CUDA(c, cudaMemsetAsync(c->d_mT, 0, kTableFloats * sizeof(float), c->stream));
    SG_CUDA(c, cudaMemsetAsync(c->d_vT, 0, kTableFloats * sizeof(float), c->stream));
    SG_CUDA(c, cudaMemsetAsync(c->d_gW, 0, kWeights * sizeof(float), c->stream));
    SG_CUDA(c, cudaMemsetAsync(c->d_gT, 0, kTableFloats * sizeof(float), c->stream));
    // bf16 copy: an Adam step with zero learning rate rounds the master weights
    SG_CUDA(c, launch_adam(c->d_W, c->d_gW, c->d_mW, c->d_vW, kWeights, 0.0f, 0.0f, 0.0f, 1.0f, 1.0f, 1.0f, c->d_Wb,
                           c->stream));
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_params = true;
    c->step = 0;
    c->enc_dirty = true;
    return LT_OK;
    LT_CATCH(ctx)
}

int sg_get_params(void *ctx, float *weights, float *table, int is_device) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !weights || !table) return LT_ERR_ARG;
    if (!c->has_params) return fail(c, LT_ERR_STATE, "no parameters (sg_set_params)");
    SG_CUDA(c, cudaSetDevice(c->device));
    int rc = copy_to(c, weights, c->d_W, kWeights * sizeof(float), is_device);
    if (rc) return rc;
    return copy_to(c, table, c->d_table, kTableFloats * sizeof(float), is_device);
    LT_CATCH(ctx)
}

int sg_set_training_data(void *ctx, const lt_light *lights, int32_t n_solves, const float *E_obs) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !lights || !E_obs || n_solves <= 0) return LT_ERR_ARG;
    if (!c->n) return fail(c, LT_ERR_STATE, "no texels (sg_set_texels)");
    std::vector<LightC> L;
    int rc = derive(c, lights, n_solves, &L);
    if (rc) return rc;
    SG_CUDA(c, cudaSetDevice(c->device));
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    SG_CUDA(c, dalloc(c->d_train, L.size()));
    SG_CUDA(c, cudaMemcpy(c->d_train, L.data(), L.size() * sizeof(LightC), cudaMemcpyHostToDevice));
    c->n_solves = n_solves;
    c->E_obs = E_obs;
    return LT_OK;
    LT_CATCH(ctx)
}

static int check_device(SgCtx *c);

int sg_train_step(void *ctx, uint64_t seed, int32_t batch, float lr, const int32_t *samples, double *loss_out) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c) return LT_ERR_ARG;
    int rc = need_params(c);
    if (rc) return rc;
    if (!c->n_solves) return fail(c, LT_ERR_STATE, "no training data (sg_set_training_data)");
    if (batch < 1 || batch > SG_MAX_BATCH) return fail(c, LT_ERR_ARG, "batch must be in [1, SG_MAX_BATCH]");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return fail(c, LT_ERR_ARG, "learning rate must be finite and >= 0");
    SG_CUDA(c, cudaSetDevice(c->device));
    if ((rc = ensure_rows(c, batch))) return rc;
    const int32_t *d_samples = nullptr;
    if (samples) {
        for (int32_t i = 0; i < batch; ++i)
            if (samples[2 * i] < 0 || samples[2 * i] >= c->n_solves || samples[2 * i + 1] < 0 ||
                (int64_t)samples[2 * i + 1] >= c->n)
                return fail(c, LT_ERR_ARG, "sample out of range");
        size_t cap = (size_t)c->samples_cap;
        SG_CUDA(c, ensure(c->d_samples, cap, (size_t)2 * batch));
        c->samples_cap = (int32_t)cap;
        SG_CUDA(c, cudaMemcpyAsync(c->d_samples, samples, (size_t)2 * batch * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   c->stream));
        d_samples = c->d_samples;
    }
    SG_CUDA(c, cudaMemsetAsync(c->d_gT, 0, kTableFloats * sizeof(float), c->stream));
    TrainArgs a;
    a.tex = view(c);
    a.lights = c->d_train;
    a.n_solves = c->n_solves;
    a.E_obs = c->E_obs;
    a.samples = d_samples;
    a.seed = seed;
    a.step = (uint64_t)c->step;
    a.batch = batch;
    a.table = c->d_table;
    a.dtable = c->d_gT;
    a.Wb = c->d_Wb;
    a.rb = c->rb;
    a.loss_part = c->d_lpart;
    int grid = 0;
    if (c->train_tc) {
        SG_CUDA(c, launch_train_tc(a, c->d_err, c->stream, &grid));
    } else {
        const int64_t tiles = ((int64_t)batch + 15) / 16;
        grid = (int)std::min<int64_t>((tiles + kMlpWarps - 1) / kMlpWarps, train_grid(c->device));
        SG_CUDA(c, launch_train(a, grid, c->stream));
    }
    SG_CUDA(c, launch_wgrad(c->rb, batch, c->d_wpart, c->d_gW, c->d_lpart, grid, c->d_loss, c->stream));
    ++c->step;
    const double b1 = 0.9, b2 = 0.99;
    const float bc1 = (float)(1.0 - std::pow(b1, (double)c->step));
    const float bc2 = (float)(1.0 - std::pow(b2, (double)c->step));
    SG_CUDA(c, launch_adam(c->d_W, c->d_gW, c->d_mW, c->d_vW, kWeights, lr, (float)b1, (float)b2, 1e-15f, bc1, bc2,
                           c->d_Wb, c->stream));
    SG_CUDA(c, launch_adam(c->d_table, c->d_gT, c->d_mT, c->d_vT, kTableFloats, lr, (float)b1, (float)b2, 1e-15f, bc1,
                           bc2, nullptr, c->stream));
    c->enc_dirty = true;
    if (loss_out) {
        SG_CUDA(c, cudaMemcpyAsync(loss_out, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        return check_device(c);   // synchronises; reports a tensor-core wait that gave up
    }
    return LT_OK;
    LT_CATCH(ctx)
}

int sg_get_gradients(void *ctx, float *dweights, float *dtable, int is_device) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !dweights || !dtable) return LT_ERR_ARG;
    SG_CUDA(c, cudaSetDevice(c->device));
    int rc = copy_to(c, dweights, c->d_gW, kWeights * sizeof(float), is_device);
    if (rc) return rc;
    return copy_to(c, dtable, c->d_gT, kTableFloats * sizeof(float), is_device);
    LT_CATCH(ctx)
}

static int design_prepare(SgCtx *c, const lt_light *lights, int32_t n_lights) {
    std::vector<LightC> L;
    int rc = derive(c, lights, n_lights, &L);
    if (rc) return rc;
    if (c->dl_cap < n_lights) {
        SG_CUDA(c, cudaStreamSynchronize(c->stream));
        SG_CUDA(c, dalloc(c->d_dl, (size_t)n_lights));
        c->dl_cap = n_lights;
    }
    if ((rc = ensure_pinned(c, (size_t)n_lights * sizeof(LightC) + ((size_t)n_lights * 8 + 8) * sizeof(double))))
        return rc;
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    std::memcpy(c->h_pinned, L.data(), L.size() * sizeof(LightC));
    SG_CUDA(c, cudaMemcpyAsync(c->d_dl, c->h_pinned, L.size() * sizeof(LightC), cudaMemcpyHostToDevice, c->stream));
    SG_CUDA(c, ensure(c->d_K, c->K_floats, (size_t)n_lights * (size_t)c->n_pad));
    return refresh_encoding(c);
}

static int forward_rows(SgCtx *c, const DesignArgs &a) {
    if (c->use_tc) SG_CUDA(c, launch_design_forward_tc(a, c->d_err, c->stream));
    else SG_CUDA(c, launch_design_forward(a, c->stream));
    return LT_OK;
}

// Reads and clears the device error word (synchronises the stream).
static int check_device(SgCtx *c) {
    int32_t e = 0;
    SG_CUDA(c, cudaMemcpyAsync(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (e) {
        SG_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream));
        return fail(c, LT_ERR_TIMEOUT, "a tensor-core wait gave up (device error word " + std::to_string(e) + ")");
    }
    return LT_OK;
}

static DesignArgs design_args(SgCtx *c, int32_t n_lights) {
    DesignArgs a;
    a.tex = view(c);
    a.lights = c->d_dl;
    a.n_lights = n_lights;
    a.enc = c->d_enc;
    a.Wb = c->d_Wb;
    a.K = c->d_K;
    a.up = c->d_up;
    a.gpart = c->d_gpart;
    return a;
}

int sg_response(void *ctx, const lt_light *light, float *K_out, int is_device) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !light || !K_out) return LT_ERR_ARG;
    int rc = need_params(c);
    if (rc) return rc;
    SG_CUDA(c, cudaSetDevice(c->device));
    if ((rc = design_prepare(c, light, 1))) return rc;
    if ((rc = forward_rows(c, design_args(c, 1)))) return rc;
    if ((rc = check_device(c))) return rc;
    return copy_to(c, K_out, c->d_K, (size_t)c->n * sizeof(float), is_device);
    LT_CATCH(ctx)
}

int sg_design(void *ctx, const lt_light *lights, int32_t n_lights, const float *E_target, const float *alpha,
              double *loss_out, double *grad_out, float *E_out) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !lights || !E_target || n_lights <= 0) return LT_ERR_ARG;
    if (n_lights > LT_MAX_LIGHTS) return fail(c, LT_ERR_ARG, "more lights than LT_MAX_LIGHTS");
    int rc = need_params(c);
    if (rc) return rc;
    SG_CUDA(c, cudaSetDevice(c->device));
    if ((rc = design_prepare(c, lights, n_lights))) return rc;
    SG_CUDA(c, ensure(c->d_up, c->up_floats, (size_t)c->n_pad));
    if (!c->d_dout) SG_CUDA(c, dalloc(c->d_dout, (size_t)LT_MAX_LIGHTS * 8 + 8));
    if (c->use_tc && n_lights <= kFusedMaxLights) {
        // one kernel: forward, per-texel irradiance and weights, backward
        FusedArgs f;
        f.target = E_target;
        f.alpha = alpha;
        f.E_out = E_out;
        f.loss_part = c->d_lpart;
        f.texels_per_tile = 128 / n_lights;
        f.n_tiles = (c->n_pad + f.texels_per_tile - 1) / f.texels_per_tile;
        SG_CUDA(c, ensure(c->d_gpart, c->gpart_floats, (size_t)n_lights * (size_t)f.n_tiles * 8));
        const DesignArgs a = design_args(c, n_lights);
        int grid = 0;
        SG_CUDA(c, launch_design_fused_tc(a, f, c->d_err, c->stream, &grid));
        SG_CUDA(c, launch_design_final(c->d_gpart, c->d_dl, n_lights, f.n_tiles, c->d_lpart, grid, c->d_dout,
                                       c->stream));
    } else {
        const int64_t tpl = c->n_pad / 16;
        SG_CUDA(c, ensure(c->d_gpart, c->gpart_floats, (size_t)n_lights * (size_t)tpl * 8));
        const DesignArgs a = design_args(c, n_lights);
        if ((rc = forward_rows(c, a))) return rc;
        SG_CUDA(c, launch_design_reduce(a.tex, c->d_dl, n_lights, c->d_K, E_target, alpha, E_out, c->d_up,
                                        c->d_lpart, c->stream));
        if (c->use_tc) SG_CUDA(c, launch_design_backward_tc(a, c->d_err, c->stream));
        else SG_CUDA(c, launch_design_backward(a, c->stream));
        SG_CUDA(c, launch_design_final(c->d_gpart, c->d_dl, n_lights, tpl, c->d_lpart, 0, c->d_dout, c->stream));
    }
    double *h = c->h_pinned + (n_lights * sizeof(LightC) + sizeof(double) - 1) / sizeof(double);
    SG_CUDA(c, cudaMemcpyAsync(h, c->d_dout, ((size_t)n_lights * 8 + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    if ((rc = check_device(c))) return rc;
    if (grad_out) std::memcpy(grad_out, h, (size_t)n_lights * 8 * sizeof(double));
    if (loss_out) *loss_out = h[(size_t)n_lights * 8];
    return LT_OK;
    LT_CATCH(ctx)
}

int sg_network(void *ctx, const float *X, int32_t rows, const float *dO, float *O_out, float *dX_out, float *dW_out) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !X || !O_out || rows <= 0 || rows > SG_MAX_BATCH) return LT_ERR_ARG;
    if (!c->has_params) return fail(c, LT_ERR_STATE, "no parameters (sg_set_params)");
    SG_CUDA(c, cudaSetDevice(c->device));
    int rc = ensure_rows(c, rows);
    if (rc) return rc;
    const size_t need = (size_t)rows * 64;
    if (c->scratch_floats < need) {
        SG_CUDA(c, cudaStreamSynchronize(c->stream));
        SG_CUDA(c, dalloc(c->d_X, need));
        SG_CUDA(c, dalloc(c->d_dX, need));
        SG_CUDA(c, dalloc(c->d_dO, need / 4));
        SG_CUDA(c, dalloc(c->d_O, need / 4));
        SG_CUDA(c, dalloc(c->d_xn, need));
        SG_CUDA(c, dalloc(c->d_enc_out, need));
        c->scratch_floats = need;
    }
    SG_CUDA(c, cudaMemcpyAsync(c->d_X, X, need * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    if (dO)
        SG_CUDA(c, cudaMemcpyAsync(c->d_dO, dO, (size_t)rows * 16 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    NetworkArgs a;
    a.X = c->d_X;
    a.dO = dO ? c->d_dO : nullptr;
    a.rows = rows;
    a.Wb = c->d_Wb;
    a.O = c->d_O;
    a.dX = dO ? c->d_dX : nullptr;
    a.rb = c->rb;
    SG_CUDA(c, launch_network(a, c->stream));
    if (dO && dW_out) {
        SG_CUDA(c, launch_wgrad(c->rb, rows, c->d_wpart, c->d_gW, nullptr, 0, nullptr, c->stream));
        SG_CUDA(c, cudaMemcpyAsync(dW_out, c->d_gW, kWeights * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    SG_CUDA(c, cudaMemcpyAsync(O_out, c->d_O, (size_t)rows * 16 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (dO && dX_out)
        SG_CUDA(c, cudaMemcpyAsync(dX_out, c->d_dX, need * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    return LT_OK;
    LT_CATCH(ctx)
}

int sg_set_kernels(void *ctx, int flags) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || (flags & ~(SG_KERNELS_DESIGN_TC | SG_KERNELS_TRAIN_TC))) return LT_ERR_ARG;
    c->use_tc = (flags & SG_KERNELS_DESIGN_TC) ? 1 : 0;
    c->train_tc = (flags & SG_KERNELS_TRAIN_TC) ? 1 : 0;
    return LT_OK;
    LT_CATCH(ctx)
}

int sg_encode(void *ctx, const float *xn, int32_t rows, float *enc_out) {
    LT_TRY
    SgCtx *c = static_cast<SgCtx *>(ctx);
    if (!c || !xn || !enc_out || rows <= 0 || rows > SG_MAX_BATCH) return LT_ERR_ARG;
    if (!c->has_params) return fail(c, LT_ERR_STATE, "no parameters (sg_set_params)");
    SG_CUDA(c, cudaSetDevice(c->device));
    const size_t need = (size_t)rows * 64;
    if (c->scratch_floats < need) {
        SG_CUDA(c, cudaStreamSynchronize(c->stream));
        SG_CUDA(c, dalloc(c->d_X, need));
        SG_CUDA(c, dalloc(c->d_dX, need));
        SG_CUDA(c, dalloc(c->d_dO, need / 4));
        SG_CUDA(c, dalloc(c->d_O, need / 4));
        SG_CUDA(c, dalloc(c->d_xn, need));
        SG_CUDA(c, dalloc(c->d_enc_out, need));
        c->scratch_floats = need;
    }
    SG_CUDA(c, cudaMemcpyAsync(c->d_xn, xn, (size_t)rows * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    SG_CUDA(c, launch_encode_points(c->d_xn, rows, c->d_table, c->d_enc_out, c->stream));
    SG_CUDA(c, cudaMemcpyAsync(enc_out, c->d_enc_out, (size_t)rows * 32 * sizeof(float), cudaMemcpyDeviceToHost,
                               c->stream));
    SG_CUDA(c, cudaStreamSynchronize(c->stream));
    return LT_OK;
    LT_CATCH(ctx)
}

}  // extern "C"
