/*
 * oracle.c -- plain, slow CPU oracle for view-independent adjoint light tracing.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline and reference legs load this library. The product path (the CUDA
 * library and its Python binding) never calls it, shares no code with it and
 * fails when its own extension is missing.
 *
 * What it computes, following Lipp et al., "View-Independent Adjoint Light
 * Tracing for Lighting Design Optimization" (arXiv 2310.02043):
 *   - Alg. 1 (primal light tracing) with the indirect-flux recursion of Eq. 7,
 *     specialised to Lambertian surfaces and cosine-weighted bounces, and the
 *     coefficient update of Eq. 8 / Eq. S.9 for order n = 0 with a per-texel
 *     box basis: every hit adds Phi_i / A_t to the irradiance E_t of the texel
 *     it lands in.
 *   - Alg. 2 (adjoint light tracing): the same paths replayed from the same
 *     random numbers; the adjoint state dO/dPhi_r of Eq. 12 is summed along the
 *     path and multiplied with dPhi_r/dp (Eq. 11). For Lambertian BRDFs the BRDF
 *     adjoints of Eq. 13 vanish.
 *   - dPhi_r/dp of Sec. 4.4 and the supplement: intensity I_e = p^2/2, the
 *     "virtual intensity" position derivative (Eq. 14, with the cos/r^2
 *     gradient that Alg. S1 derives, regulariser 0), the spot soft edge a(theta)
 *     of Eq. S.11 and its position term (Eq. S.12), and the orientation chain
 *     rule (Eq. 15) with a yaw/pitch axis instead of a rotation vector.
 *   - Rectangular area lights (supplement, Eq. S.15-S.16): a Lambertian
 *     rectangle of total power P = p^2/2, rays sampled uniformly over its
 *     surface and over the hemisphere about its normal, Phi_r = 2 P cos / N
 *     (expected total P); dPhi_r/dp = Phi_r d log(cos_1 / r^2) + Phi_r
 *     d log(cos theta), with the first hit fixed and the ray origin moving
 *     rigidly with the light (translation, and rotation about the centroid).
 *
 * Precision: everything continuous (flux, hit points, directions, derivatives,
 * sums) is double. The two integer decisions of every segment -- which
 * triangle is hit first and which texel the hit falls in -- are taken in
 * float, the precision the GPU path takes them in: the ray is rounded to
 * float and tested with the watertight ray/triangle test of Woop, Benthin and
 * Wald (JCGT 2013), closest hit by brute force over all triangles (ties go
 * to the lower triangle index).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC 2011), counter =
 * (photon index low, photon index high, segment, design word), key = (seed
 * low, seed high); uniform u = (x >> 8) * 2^-24 from counter lanes 0 and 1
 * (directions), and from lanes 2 and 3 for the position on an area light.
 *
 * Build: plain C99 with OpenMP; compile with -ffp-contract=off so float
 * arithmetic is the same on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies with the */
/* published multipliers and Weyl key increments.                             */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four uniforms in [0, 1) for (photon, segment, design) under `seed`. */
static void draw4(uint64_t seed, uint64_t photon, uint32_t segment, uint32_t design, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)photon, (uint32_t)(photon >> 32), segment, design};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    for (int k = 0; k < 4; ++k) u[k] = (double)(r[k] >> 8) * (1.0 / 16777216.0);
}

/* The first two of them. */
static void draw2(uint64_t seed, uint64_t photon, uint32_t segment, uint32_t design, double *u1, double *u2)
{
    double u[4];
    draw4(seed, photon, segment, design, u);
    *u1 = u[0];
    *u2 = u[1];
}

/* ------------------------------------------------------------------------ */
/* Small vector helpers (double)                                             */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------------ */
/* Scene                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n_tri;
    const float *xyz;       /* [n_tri][3][3] */
    const float *uv;        /* [n_tri][3][2] */
    const int32_t *tile;    /* [n_tri] */
    const float *albedo;    /* [n_tri] */
    int32_t n_tiles;
    const int32_t *res;     /* [n_tiles][2] */
    const double *tile_area;/* [n_tiles] */
    int64_t *tile_off;      /* [n_tiles + 1], owned */
    double *texel_area;     /* [n_texels], owned: A_t = tile area / (res_u res_v) */
    int64_t n_texels;
} or_scene;

static int scene_init(or_scene *s, const float *xyz, const float *uv, const int32_t *tile, const float *albedo,
                      int32_t n_tri, const int32_t *res, const double *tile_area, int32_t n_tiles)
{
    s->n_tri = n_tri; s->xyz = xyz; s->uv = uv; s->tile = tile; s->albedo = albedo;
    s->n_tiles = n_tiles; s->res = res; s->tile_area = tile_area;
    s->tile_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_tiles + 1));
    if (!s->tile_off) return -1;
    s->tile_off[0] = 0;
    for (int32_t k = 0; k < n_tiles; ++k)
        s->tile_off[k + 1] = s->tile_off[k] + (int64_t)res[2 * k] * (int64_t)res[2 * k + 1];
    s->n_texels = s->tile_off[n_tiles];
    s->texel_area = (double *)malloc(sizeof(double) * (size_t)(s->n_texels > 0 ? s->n_texels : 1));
    if (!s->texel_area) { free(s->tile_off); return -1; }
    for (int32_t k = 0; k < n_tiles; ++k) {
        double a = tile_area[k] / ((double)res[2 * k] * (double)res[2 * k + 1]);
        for (int64_t t = s->tile_off[k]; t < s->tile_off[k + 1]; ++t) s->texel_area[t] = a;
    }
    return 0;
}

static void scene_free(or_scene *s)
{
    free(s->tile_off);
    free(s->texel_area);
}

/* ------------------------------------------------------------------------ */
/* Watertight ray/triangle test in float (Woop, Benthin, Wald, JCGT 2013).   */
/* The ray is sheared so that it runs along +z; the three 2-D edge functions */
/* decide inside/outside, falling back to double when one of them is zero.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    float org[3];
    int kx, ky, kz;
    float Sx, Sy, Sz;
} or_fray;

static void fray_init(or_fray *r, const double o[3], const double d[3])
{
    float df[3];
    for (int k = 0; k < 3; ++k) { r->org[k] = (float)o[k]; df[k] = (float)d[k]; }
    int kz = 0;
    if (fabsf(df[1]) > fabsf(df[kz])) kz = 1;
    if (fabsf(df[2]) > fabsf(df[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (df[kz] < 0.0f) { int tmp = kx; kx = ky; ky = tmp; }
    r->kx = kx; r->ky = ky; r->kz = kz;
    r->Sx = df[kx] / df[kz];
    r->Sy = df[ky] / df[kz];
    r->Sz = 1.0f / df[kz];
}

/* Returns 1 on a hit with t > 0; writes t and the barycentric weights of the
 * three vertices (b0 for vertex 0, ...), all in float. */
static int fray_triangle(const or_fray *r, const float *v, float *t_out, float b_out[3])
{
    const int kx = r->kx, ky = r->ky, kz = r->kz;
    float A[3], B[3], C[3];
    for (int k = 0; k < 3; ++k) {
        A[k] = v[0 + k] - r->org[k];
        B[k] = v[3 + k] - r->org[k];
        C[k] = v[6 + k] - r->org[k];
    }
    float Ax = A[kx] - r->Sx * A[kz], Ay = A[ky] - r->Sy * A[kz];
    float Bx = B[kx] - r->Sx * B[kz], By = B[ky] - r->Sy * B[kz];
    float Cx = C[kx] - r->Sx * C[kz], Cy = C[ky] - r->Sy * C[kz];
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;
    float det = U + V + W;
    if (det == 0.0f) return 0;
    float Az = r->Sz * A[kz], Bz = r->Sz * B[kz], Cz = r->Sz * C[kz];
    float T = U * Az + V * Bz + W * Cz;
    if (det < 0.0f) { det = -det; T = -T; U = -U; V = -V; W = -W; }
    if (!(T > 0.0f)) return 0;
    *t_out = T / det;
    b_out[0] = U / det;
    b_out[1] = V / det;
    b_out[2] = W / det;
    return 1;
}

typedef struct {
    int32_t tri;    /* -1 on a miss */
    float t;
    float b[3];
} or_hit;

/* Closest hit over all triangles except those of tile `skip_tile` (the planar
 * tile the ray leaves). Ties in t go to the lower triangle index. */
static or_hit closest_hit(const or_scene *s, const double o[3], const double d[3], int32_t skip_tile)
{
    or_fray r;
    fray_init(&r, o, d);
    or_hit best;
    best.tri = -1; best.t = INFINITY;
    best.b[0] = best.b[1] = best.b[2] = 0.0f;
    for (int32_t i = 0; i < s->n_tri; ++i) {
        if (s->tile[i] == skip_tile) continue;
        float t, b[3];
        if (!fray_triangle(&r, s->xyz + 9 * (size_t)i, &t, b)) continue;
        if (t < best.t) {
            best.tri = i; best.t = t;
            best.b[0] = b[0]; best.b[1] = b[1]; best.b[2] = b[2];
        }
    }
    return best;
}

/* Texel of a hit: chart coordinates interpolated in float from the
 * barycentric weights, clamped to [0, 1], index min(floor(u res), res - 1). */
static int64_t texel_of(const or_scene *s, const or_hit *h)
{
    const float *uv = s->uv + 6 * (size_t)h->tri;
    float u = h->b[0] * uv[0] + h->b[1] * uv[2] + h->b[2] * uv[4];
    float v = h->b[0] * uv[1] + h->b[1] * uv[3] + h->b[2] * uv[5];
    u = u < 0.0f ? 0.0f : (u > 1.0f ? 1.0f : u);
    v = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
    int32_t tile = s->tile[h->tri];
    int32_t ru = s->res[2 * tile], rv = s->res[2 * tile + 1];
    int32_t iu = (int32_t)floorf(u * (float)ru);
    int32_t iv = (int32_t)floorf(v * (float)rv);
    if (iu > ru - 1) iu = ru - 1;
    if (iv > rv - 1) iv = rv - 1;
    if (iu < 0) iu = 0;
    if (iv < 0) iv = 0;
    return s->tile_off[tile] + (int64_t)iu + (int64_t)ru * (int64_t)iv;
}

/* Unit geometric normal of a triangle, double. */
static void tri_normal(const or_scene *s, int32_t tri, double n[3])
{
    const float *v = s->xyz + 9 * (size_t)tri;
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) { e1[k] = (double)v[3 + k] - v[k]; e2[k] = (double)v[6 + k] - v[k]; }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double l = norm3(n);
    n[0] /= l; n[1] /= l; n[2] /= l;
}

/* ------------------------------------------------------------------------ */
/* Luminaires (Sec. 4.4, supplement "Derivative terms")                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int type;               /* 0 point, 1 spot, 2 rectangular area light */
    double x[3];
    double yaw, pitch, p, th_in, th_out;
    double I;               /* I_e = p^2 / 2 (Sec. 4.4.1) */
    double ns[3];           /* spot axis n(yaw, pitch) */
    double e1[3], e2[3];    /* dn/dpitch and dn/dyaw / cos(pitch): frame around n */
    double dn_dyaw[3], dn_dpitch[3];
    double co, ci;          /* cos(theta_out), cos(theta_in) */
    double omega;           /* flux per ray = I omega a / N: 4 pi (point), 2 pi (1 - cos theta_out) (spot),
                               2 (area: Phi_r = 2 P cos / N with a = cos) */
    double t[3], b[3];      /* area: rectangle edges' directions, t = dn/dpitch, b = n x t */
    double half_u, half_v;  /* area: half width along t, half height along b */
    uint64_t n_rays;        /* N_l */
    uint64_t first;         /* first global photon index of this light */
} or_light;

/* The photon budget is split evenly over the lights; the first N mod L lights
 * take one extra ray. */
static void lights_init(or_light *L, const double *params, int32_t n_lights, uint64_t n_photons)
{
    uint64_t base = n_photons / (uint64_t)n_lights, rem = n_photons % (uint64_t)n_lights;
    uint64_t first = 0;
    for (int32_t l = 0; l < n_lights; ++l) {
        const double *q = params + 9 * (size_t)l;
        or_light *o = &L[l];
        memset(o, 0, sizeof(*o));
        o->type = (int)q[0];
        o->x[0] = q[1]; o->x[1] = q[2]; o->x[2] = q[3];
        o->yaw = q[4]; o->pitch = q[5]; o->p = q[6]; o->th_in = q[7]; o->th_out = q[8];
        o->I = 0.5 * o->p * o->p;
        double cy = cos(o->yaw), sy = sin(o->yaw), cp = cos(o->pitch), sp = sin(o->pitch);
        o->ns[0] = cp * cy; o->ns[1] = cp * sy; o->ns[2] = sp;
        o->dn_dyaw[0] = -cp * sy; o->dn_dyaw[1] = cp * cy; o->dn_dyaw[2] = 0.0;
        o->dn_dpitch[0] = -sp * cy; o->dn_dpitch[1] = -sp * sy; o->dn_dpitch[2] = cp;
        o->e1[0] = -sp * cy; o->e1[1] = -sp * sy; o->e1[2] = cp;
        o->e2[0] = -sy; o->e2[1] = cy; o->e2[2] = 0.0;
        if (o->type == 1) {
            o->co = cos(o->th_out);
            o->ci = cos(o->th_in);
            o->omega = 2.0 * OR_PI * (1.0 - o->co);
        } else if (o->type == 2) {
            /* the theta_in / theta_out slots carry the width and height */
            o->co = 0.0;
            o->omega = 2.0;
            o->half_u = 0.5 * o->th_in;
            o->half_v = 0.5 * o->th_out;
            for (int k = 0; k < 3; ++k) o->t[k] = o->e1[k];
            o->b[0] = sy; o->b[1] = -cy; o->b[2] = 0.0;
        } else {
            o->omega = 4.0 * OR_PI;
        }
        o->n_rays = base + ((uint64_t)l < rem ? 1u : 0u);
        o->first = first;
        first += o->n_rays;
    }
}

static int32_t light_of(const or_light *L, int32_t n_lights, uint64_t photon)
{
    for (int32_t l = 0; l < n_lights; ++l)
        if (photon < L[l].first + L[l].n_rays) return l;
    return n_lights - 1;
}

/* Quadratic soft edge of a spot in terms of cos(theta) (Eq. S.11). */
static double spot_falloff(const or_light *L, double c)
{
    if (c >= L->ci) return 1.0;
    if (c <= L->co) return 0.0;
    double s = (c - L->co) / (L->ci - L->co);
    return s * s;
}

/* Exitant ray of a light: origin x0, direction w and flux Phi_r (Sec. 4.2
 * and the supplement: point lights sample the sphere uniformly,
 * Phi_r = I 4 pi / N; spots sample the outer cone uniformly,
 * Phi_r = I 2 pi (1 - cos theta_out) a / N; area lights sample their
 * rectangle (u3, u4) and the hemisphere about n uniformly, Phi_r =
 * 2 P cos theta / N). */
static double emit(const or_light *L, const double u[4], double x0[3], double w[3], double *a_out)
{
    double u1 = u[0], u2 = u[1];
    double phi = 2.0 * OR_PI * u2;
    for (int k = 0; k < 3; ++k) x0[k] = L->x[k];
    if (L->type == 2) {
        double c = 1.0 - u1;
        double s = sqrt(fmax(0.0, 1.0 - c * c));
        double su = (2.0 * u[2] - 1.0) * L->half_u, sv = (2.0 * u[3] - 1.0) * L->half_v;
        for (int k = 0; k < 3; ++k) {
            w[k] = s * cos(phi) * L->e1[k] + s * sin(phi) * L->e2[k] + c * L->ns[k];
            x0[k] = L->x[k] + su * L->t[k] + sv * L->b[k];
        }
        *a_out = c;
        return L->I * L->omega * c / (double)L->n_rays;
    }
    if (L->type == 1) {
        double c = 1.0 - u1 * (1.0 - L->co);
        double s = sqrt(fmax(0.0, 1.0 - c * c));
        for (int k = 0; k < 3; ++k)
            w[k] = s * cos(phi) * L->e1[k] + s * sin(phi) * L->e2[k] + c * L->ns[k];
        double a = spot_falloff(L, c);
        *a_out = a;
        return L->I * L->omega * a / (double)L->n_rays;
    }
    double c = 1.0 - 2.0 * u1;
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    w[0] = s * cos(phi); w[1] = s * sin(phi); w[2] = c;
    *a_out = 1.0;
    return L->I * L->omega / (double)L->n_rays;
}

/* Cosine-weighted direction about the unit normal n (Alg. 1, "cos-weighted
 * random in H^2"), through the branchless orthonormal basis of Duff et al.
 * (JCGT 2017). */
static void cosine_dir(const double n[3], double u1, double u2, double w[3])
{
    double sgn = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    double t1[3] = {1.0 + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0]};
    double t2[3] = {b, sgn + n[1] * n[1] * a, -n[1]};
    double r = sqrt(u1), phi = 2.0 * OR_PI * u2, z = sqrt(1.0 - u1);
    double lx = r * cos(phi), ly = r * sin(phi);
    for (int k = 0; k < 3; ++k) w[k] = lx * t1[k] + ly * t2[k] + z * n[k];
}

static void area_dflux(const or_light *L, double phi_r, const double x0[3], double su, double sv,
                       const double x1[3], const double n1[3], double out[8]);

/* dPhi_r/dp at the first hit x1 with the first hit held fixed (Sec. 4.4.2).
 * n1 is the unit normal at x1 facing the light; x0 the ray origin and
 * (su, sv) its coordinates on an area light. Output order:
 * [x, y, z, yaw, pitch, p_int, theta_in, theta_out]. */
static void dflux_dp(const or_light *L, double phi_r, double a_emit, const double x0[3], double su, double sv,
                     const double x1[3], const double n1[3], double out[8])
{
    for (int k = 0; k < 8; ++k) out[k] = 0.0;
    if (L->type == 2) {
        area_dflux(L, phi_r, x0, su, sv, x1, n1, out);
        return;
    }
    double d[3] = {L->x[0] - x1[0], L->x[1] - x1[1], L->x[2] - x1[2]};
    double ell = norm3(d);
    double u[3] = {d[0] / ell, d[1] / ell, d[2] / ell};
    double c1 = dot3(n1, u);
    /* Eq. 14: dPhi/dx = I~ d(cos/r^2)/dx with I~ = Phi_r r^2 / cos; the
     * gradient of (n1 . d) / |d|^3 w.r.t. the light position is
     * (n1 - 3 (n1 . u) u) / |d|^3. */
    if (c1 > 0.0) {
        double It = phi_r * ell * ell / c1;
        for (int k = 0; k < 3; ++k) out[k] = It * (n1[k] - 3.0 * c1 * u[k]) / (ell * ell * ell);
    }
    /* Sec. 4.4.1: I_e = p^2/2, so dPhi_r/dp = p * (solid angle per ray) * a. */
    out[5] = L->p * L->omega * a_emit / (double)L->n_rays;
    if (L->type != 1) return;
    /* Spot soft edge (Eq. S.11-S.12): theta is the angle between the axis n
     * and the direction from the light to the fixed hit x1. */
    double wv[3] = {-u[0], -u[1], -u[2]};
    double c = dot3(L->ns, wv);
    if (!(c > L->co && c < L->ci)) return;
    double D = L->ci - L->co;
    double scale = L->I * L->omega / (double)L->n_rays;
    double da_dc = 2.0 * (c - L->co) / (D * D);
    for (int k = 0; k < 3; ++k) {
        double dc_dx = -(L->ns[k] - c * wv[k]) / ell;
        out[k] += scale * da_dc * dc_dx;
    }
    /* Eq. 15 with n(yaw, pitch): dPhi/dangle = dPhi/dn . dn/dangle, and
     * d cos(theta)/dn = w. */
    out[3] = scale * da_dc * dot3(wv, L->dn_dyaw);
    out[4] = scale * da_dc * dot3(wv, L->dn_dpitch);
    /* Cone angles through a only; the solid angle per ray is the sampling
     * measure and is held fixed with the path. */
    out[6] = scale * 2.0 * (c - L->co) * (c - L->co) * sin(L->th_in) / (D * D * D);
    out[7] = scale * (-2.0) * (c - L->co) * (c - L->ci) * sin(L->th_out) / (D * D * D);
}

/* Area light (Eq. S.15-S.16): Phi_r = 2 P cos(theta) / N with cos(theta) =
 * n . w, w the unit direction from the origin x0 to the fixed hit x1. With
 * the sampling measure held fixed, dPhi_r/dq = I~ d(cos_1 / r^2)/dq +
 * (2 P / N) d cos(theta)/dq. The origin moves rigidly with the light:
 * dx0/dx = 1, dx0/dangle = su dt/dangle + sv db/dangle, and n turns with
 * the angles. */
static void area_dflux(const or_light *L, double phi_r, const double x0[3], double su, double sv,
                       const double x1[3], const double n1[3], double out[8])
{
    double d[3] = {x0[0] - x1[0], x0[1] - x1[1], x0[2] - x1[2]};
    double ell = norm3(d);
    double u[3] = {d[0] / ell, d[1] / ell, d[2] / ell};       /* from x1 towards x0 */
    double w[3] = {-u[0], -u[1], -u[2]};                         /* emitted direction */
    double c1 = dot3(n1, u);
    double ct = dot3(L->ns, w);
    double k = L->I * L->omega / (double)L->n_rays;              /* 2 P / N */
    double g0[3] = {0.0, 0.0, 0.0};                              /* dPhi_r / dx0 */
    if (c1 > 0.0) {
        double It = phi_r * ell * ell / c1;
        for (int i = 0; i < 3; ++i) g0[i] = It * (n1[i] - 3.0 * c1 * u[i]) / (ell * ell * ell);
    }
    /* cos(theta) = -n . u: d/dx0 = -(n - (n . u) u) / r = -(n + ct u) / r */
    for (int i = 0; i < 3; ++i) g0[i] += k * (-(L->ns[i] + ct * u[i]) / ell);
    for (int i = 0; i < 3; ++i) out[i] = g0[i];
    double cy = cos(L->yaw), sy = sin(L->yaw), cp = cos(L->pitch), sp = sin(L->pitch);
    double dt_dyaw[3] = {sp * sy, -sp * cy, 0.0}, dt_dpitch[3] = {-cp * cy, -cp * sy, -sp};
    double db_dyaw[3] = {cy, sy, 0.0};
    double dx0_dyaw[3], dx0_dpitch[3];
    for (int i = 0; i < 3; ++i) {
        dx0_dyaw[i] = su * dt_dyaw[i] + sv * db_dyaw[i];
        dx0_dpitch[i] = su * dt_dpitch[i];
    }
    out[3] = dot3(g0, dx0_dyaw) + k * dot3(w, L->dn_dyaw);
    out[4] = dot3(g0, dx0_dpitch) + k * dot3(w, L->dn_dpitch);
    out[5] = L->p * L->omega * ct / (double)L->n_rays;           /* P = p^2 / 2 */
}

/* ------------------------------------------------------------------------ */
/* One photon path (Alg. 1 / Alg. 2)                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t texel;
    double phi;     /* incident flux Phi_i deposited */
} or_deposit;

typedef struct {
    /* forward */
    or_deposit *dep; int n_dep;
    /* adjoint */
    const double *w;        /* dO/dE_t * (1/A_t) * A_t = alpha_t (E_t - E*_t), per texel */
    double grad[8]; int has_grad;
    /* path record */
    int32_t *rec_tri; int64_t *rec_texel;
    double *rec_phi;        /* flux Phi_i deposited at each hit (may be NULL) */
    uint64_t segments;
} or_path_io;

static void trace_photon(const or_scene *s, const or_light *L, int32_t n_lights, uint64_t seed, uint32_t design,
                         uint64_t photon, int32_t max_hits, or_path_io *io)
{
    int32_t l = light_of(L, n_lights, photon);
    const or_light *lt = &L[l];
    double u1, u2, w[3], a_emit, u0[4], o[3];
    draw4(seed, photon, 0u, design, u0);
    double phi_r = emit(lt, u0, o, w, &a_emit);
    double phi = phi_r;
    double x0[3] = {o[0], o[1], o[2]};
    double su = (2.0 * u0[2] - 1.0) * lt->half_u, sv = (2.0 * u0[3] - 1.0) * lt->half_v;
    int32_t skip_tile = -1;
    double g = 0.0, beta = 1.0, dphi[8];
    io->has_grad = 0;
    for (int32_t i = 1; i <= max_hits; ++i) {
        or_hit h = closest_hit(s, o, w, skip_tile);
        io->segments += 1;
        if (h.tri < 0) break;
        double x[3];
        for (int k = 0; k < 3; ++k) x[k] = o[k] + (double)h.t * w[k];
        int64_t t = texel_of(s, &h);
        double n[3];
        tri_normal(s, h.tri, n);
        if (dot3(n, w) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        if (io->rec_tri) { io->rec_tri[i - 1] = h.tri; io->rec_texel[i - 1] = t; }
        if (io->rec_phi) io->rec_phi[i - 1] = phi;
        if (io->dep) {                                  /* Eq. 8, n = 0 box basis */
            io->dep[io->n_dep].texel = t;
            io->dep[io->n_dep].phi = phi;
            io->n_dep += 1;
        }
        if (io->w) {
            if (i == 1) { dflux_dp(lt, phi_r, a_emit, x0, su, sv, x, n, dphi); io->has_grad = 1; }
            g += io->w[t] * beta;                       /* Eq. 12 */
        }
        if (i == max_hits) break;
        double rho = (double)s->albedo[h.tri];
        draw2(seed, photon, (uint32_t)i, design, &u1, &u2);
        cosine_dir(n, u1, u2, w);
        phi *= rho;                                     /* Eq. 7: f cos / p = rho */
        beta *= rho;
        o[0] = x[0]; o[1] = x[1]; o[2] = x[2];
        skip_tile = s->tile[h.tri];
    }
    if (io->w && io->has_grad)
        for (int k = 0; k < 8; ++k) io->grad[k] = g * dphi[k];  /* Eq. 11 */
}

/* ------------------------------------------------------------------------ */
/* Exported passes. Photons are processed in fixed chunks; results are       */
/* merged in photon order, so sums do not depend on the thread count.        */
/* ------------------------------------------------------------------------ */
#define OR_CHUNK 512

static int threads_of(int n_threads)
{
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

int or_texel_count(const int32_t *res, int32_t n_tiles, int64_t *out)
{
    int64_t n = 0;
    for (int32_t k = 0; k < n_tiles; ++k) n += (int64_t)res[2 * k] * res[2 * k + 1];
    *out = n;
    return 0;
}

/* Forward pass (Alg. 1) over photons [begin, end) of an n_photons budget.
 * E accumulates irradiance per texel (caller zeroes it); count (may be NULL)
 * accumulates deposits per texel; stats[0] += segments, stats[1] += deposits. */
int or_forward(const float *xyz, const float *uv, const int32_t *tile, const float *albedo, int32_t n_tri,
               const int32_t *res, const double *tile_area, int32_t n_tiles,
               const double *light_params, int32_t n_lights,
               uint64_t seed, uint32_t design, uint64_t n_photons, uint64_t begin, uint64_t end, int32_t max_hits,
               double *E, int64_t *count, double *stats, int n_threads)
{
    if (n_lights <= 0 || max_hits <= 0 || end < begin || end > n_photons) return -1;
    or_scene s;
    if (scene_init(&s, xyz, uv, tile, albedo, n_tri, res, tile_area, n_tiles)) return -3;
    or_light *L = (or_light *)malloc(sizeof(or_light) * (size_t)n_lights);
    lights_init(L, light_params, n_lights, n_photons);
    int nt = threads_of(n_threads);
    int64_t n_chunks = (int64_t)((end - begin + OR_CHUNK - 1) / OR_CHUNK);
    int64_t per_round = (int64_t)nt * 4;
    or_deposit *buf = (or_deposit *)malloc(sizeof(or_deposit) * (size_t)per_round * OR_CHUNK * (size_t)max_hits);
    int *nbuf = (int *)calloc((size_t)per_round, sizeof(int));
    uint64_t *segs = (uint64_t *)calloc((size_t)per_round, sizeof(uint64_t));
    double total_seg = 0.0, total_dep = 0.0;
    for (int64_t r0 = 0; r0 < n_chunks; r0 += per_round) {
        int64_t r1 = r0 + per_round < n_chunks ? r0 + per_round : n_chunks;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
        for (int64_t c = r0; c < r1; ++c) {
            or_path_io io;
            memset(&io, 0, sizeof(io));
            io.dep = buf + (size_t)(c - r0) * OR_CHUNK * (size_t)max_hits;
            uint64_t p0 = begin + (uint64_t)c * OR_CHUNK;
            uint64_t p1 = p0 + OR_CHUNK < end ? p0 + OR_CHUNK : end;
            for (uint64_t p = p0; p < p1; ++p) trace_photon(&s, L, n_lights, seed, design, p, max_hits, &io);
            nbuf[c - r0] = io.n_dep;
            segs[c - r0] = io.segments;
        }
        for (int64_t c = r0; c < r1; ++c) {
            const or_deposit *d = buf + (size_t)(c - r0) * OR_CHUNK * (size_t)max_hits;
            for (int k = 0; k < nbuf[c - r0]; ++k) {
                E[d[k].texel] += d[k].phi / s.texel_area[d[k].texel];
                if (count) count[d[k].texel] += 1;
            }
            total_seg += (double)segs[c - r0];
            total_dep += (double)nbuf[c - r0];
        }
    }
    if (stats) { stats[0] += total_seg; stats[1] += total_dep; }
    free(buf); free(nbuf); free(segs); free(L);
    scene_free(&s);
    return 0;
}

/* Adjoint pass (Alg. 2) over photons [begin, end). w[t] = alpha_t (E_t - E*_t)
 * is dO/dPhi_i for a deposit into texel t. grad [n_lights][8] accumulates
 * dO/dp. stats[0] += segments. */
int or_adjoint(const float *xyz, const float *uv, const int32_t *tile, const float *albedo, int32_t n_tri,
               const int32_t *res, const double *tile_area, int32_t n_tiles,
               const double *light_params, int32_t n_lights,
               uint64_t seed, uint32_t design, uint64_t n_photons, uint64_t begin, uint64_t end, int32_t max_hits,
               const double *w, double *grad, double *stats, int n_threads)
{
    if (n_lights <= 0 || max_hits <= 0 || end < begin || end > n_photons) return -1;
    or_scene s;
    if (scene_init(&s, xyz, uv, tile, albedo, n_tri, res, tile_area, n_tiles)) return -3;
    or_light *L = (or_light *)malloc(sizeof(or_light) * (size_t)n_lights);
    lights_init(L, light_params, n_lights, n_photons);
    int nt = threads_of(n_threads);
    int64_t n_chunks = (int64_t)((end - begin + OR_CHUNK - 1) / OR_CHUNK);
    int64_t per_round = (int64_t)nt * 4;
    double *part = (double *)malloc(sizeof(double) * (size_t)per_round * (size_t)n_lights * 8);
    uint64_t *segs = (uint64_t *)calloc((size_t)per_round, sizeof(uint64_t));
    double total_seg = 0.0;
    for (int64_t r0 = 0; r0 < n_chunks; r0 += per_round) {
        int64_t r1 = r0 + per_round < n_chunks ? r0 + per_round : n_chunks;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
        for (int64_t c = r0; c < r1; ++c) {
            double *pg = part + (size_t)(c - r0) * (size_t)n_lights * 8;
            memset(pg, 0, sizeof(double) * (size_t)n_lights * 8);
            or_path_io io;
            memset(&io, 0, sizeof(io));
            io.w = w;
            uint64_t p0 = begin + (uint64_t)c * OR_CHUNK;
            uint64_t p1 = p0 + OR_CHUNK < end ? p0 + OR_CHUNK : end;
            for (uint64_t p = p0; p < p1; ++p) {
                trace_photon(&s, L, n_lights, seed, design, p, max_hits, &io);
                if (io.has_grad) {
                    int32_t l = light_of(L, n_lights, p);
                    for (int k = 0; k < 8; ++k) pg[8 * l + k] += io.grad[k];
                }
            }
            segs[c - r0] = io.segments;
        }
        for (int64_t c = r0; c < r1; ++c) {
            const double *pg = part + (size_t)(c - r0) * (size_t)n_lights * 8;
            for (int64_t k = 0; k < (int64_t)n_lights * 8; ++k) grad[k] += pg[k];
            total_seg += (double)segs[c - r0];
        }
    }
    if (stats) stats[0] += total_seg;
    free(part); free(segs); free(L);
    scene_free(&s);
    return 0;
}

/* Path record for photons [begin, begin + count): triangle and texel of every
 * hit (-1 after the path ends). phi_out (may be NULL) [count][max_hits]
 * receives the flux Phi_i each hit deposits (0 after the path ends). With
 * adjoint weights w (may be NULL), grad_out [count][8] receives each
 * photon's own gradient term. */
int or_paths(const float *xyz, const float *uv, const int32_t *tile, const float *albedo, int32_t n_tri,
             const int32_t *res, const double *tile_area, int32_t n_tiles,
             const double *light_params, int32_t n_lights,
             uint64_t seed, uint32_t design, uint64_t n_photons, uint64_t begin, uint64_t count, int32_t max_hits,
             int32_t *tri_out, int64_t *texel_out, double *phi_out, const double *w, double *grad_out,
             int n_threads)
{
    if (n_lights <= 0 || max_hits <= 0 || begin + count > n_photons) return -1;
    or_scene s;
    if (scene_init(&s, xyz, uv, tile, albedo, n_tri, res, tile_area, n_tiles)) return -3;
    or_light *L = (or_light *)malloc(sizeof(or_light) * (size_t)n_lights);
    lights_init(L, light_params, n_lights, n_photons);
    int nt = threads_of(n_threads);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t k = 0; k < (int64_t)count; ++k) {
        or_path_io io;
        memset(&io, 0, sizeof(io));
        io.rec_tri = tri_out + (size_t)k * max_hits;
        io.rec_texel = texel_out + (size_t)k * max_hits;
        for (int32_t i = 0; i < max_hits; ++i) { io.rec_tri[i] = -1; io.rec_texel[i] = -1; }
        if (phi_out) {
            io.rec_phi = phi_out + (size_t)k * max_hits;
            for (int32_t i = 0; i < max_hits; ++i) io.rec_phi[i] = 0.0;
        }
        io.w = w;
        trace_photon(&s, L, n_lights, seed, design, begin + (uint64_t)k, max_hits, &io);
        if (grad_out)
            for (int j = 0; j < 8; ++j) grad_out[8 * (size_t)k + j] = io.has_grad ? io.grad[j] : 0.0;
    }
    free(L);
    scene_free(&s);
    return 0;
}

/* Brute-force closest hit for a batch of rays (float decision, see above).
 * o, d: [n][3] double; outputs tri (-1 on miss), t, barycentrics [n][3]. */
int or_closest_hits(const float *xyz, int32_t n_tri, const int32_t *tile, const double *o, const double *d,
                    int64_t n, int32_t skip_tile, int32_t *tri_out, float *t_out, float *b_out)
{
    or_scene s;
    memset(&s, 0, sizeof(s));
    s.n_tri = n_tri; s.xyz = xyz; s.tile = tile;
    for (int64_t i = 0; i < n; ++i) {
        or_hit h = closest_hit(&s, o + 3 * i, d + 3 * i, skip_tile);
        tri_out[i] = h.tri;
        t_out[i] = h.t;
        b_out[3 * i] = h.b[0]; b_out[3 * i + 1] = h.b[1]; b_out[3 * i + 2] = h.b[2];
    }
    return 0;
}

/* dPhi_r/dp for a given light, emitted-ray falloff and fixed first hit; used
 * by the tests to check the derivative formulas in isolation. */
int or_dflux(const double *light_params, uint64_t n_rays, const double *x1, const double *n1, double a_emit,
             double u3, double u4, double *phi_out, double *out)
{
    or_light L;
    lights_init(&L, light_params, 1, n_rays);
    double x0[3] = {L.x[0], L.x[1], L.x[2]}, su = 0.0, sv = 0.0;
    if (L.type == 2) {    /* origin from the position uniforms; a = cos(theta) towards x1 */
        su = (2.0 * u3 - 1.0) * L.half_u;
        sv = (2.0 * u4 - 1.0) * L.half_v;
        for (int k = 0; k < 3; ++k) x0[k] = L.x[k] + su * L.t[k] + sv * L.b[k];
        double d[3] = {x1[0] - x0[0], x1[1] - x0[1], x1[2] - x0[2]};
        a_emit = dot3(L.ns, d) / norm3(d);
    }
    double phi_r = L.I * L.omega * a_emit / (double)L.n_rays;
    *phi_out = phi_r;
    dflux_dp(&L, phi_r, a_emit, x0, su, sv, x1, n1, out);
    return 0;
}

/* Emitted direction and falloff of photon `photon` under `seed` for a single
 * light with n_rays photons: used by the tests to check the sampling. */
int or_emit(const double *light_params, uint64_t n_rays, uint64_t seed, uint32_t design, uint64_t photon,
            double *w_out, double *phi_out, double *a_out, double *origin_out)
{
    or_light L;
    lights_init(&L, light_params, 1, n_rays);
    double u[4], x0[3];
    draw4(seed, photon, 0u, design, u);
    *phi_out = emit(&L, u, x0, w_out, a_out);
    if (origin_out)
        for (int k = 0; k < 3; ++k) origin_out[k] = x0[k];
    return 0;
}

/* Cosine-weighted direction about n from two given uniforms. */
int or_cosine_dir(const double *n, double u1, double u2, double *w_out)
{
    cosine_dir(n, u1, u2, w_out);
    return 0;
}
