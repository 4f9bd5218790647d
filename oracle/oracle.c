/*
 * oracle.c -- plain, slow CPU oracle for "Generate Coherent Rays Directly"
 * (Liu et al., arXiv 2310.07182).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the
 * smoke check and the benchmark's CPU baseline, never by the product path.
 *
 * It follows the paper's steps in the paper's order:
 *   Sec. 3.1  one path per pixel per sample (several samples = finer pixels); shading point
 *             = first hit; the secondary ray's direction is the exit direction.
 *   Sec. 3.3  interleaved grouping: W x H tiles, in-tile pixel numbers shuffled by a
 *             linear congruential sequence, group = shuffled number / K.
 *   Sec. 3.2  tangent-space direction reuse with three group types (diffuse: reuse one
 *             member's exit direction; glossy: unchanged; hybrid: diffuse members take the
 *             average tangent-space exit direction of the glossy/specular members).
 *   Sec. 3.1  world-space direct reuse, kept only as the ablation / negative control.
 * Next-event estimation (one light sample per non-specular shading point, shadow ray for
 * visibility) is an optional standard path-tracing estimator the paper does not discuss;
 * its readings are stated where it is implemented.
 * Intersection is a plain Moller-Trumbore test in FP64 over a median-split BVH (or all
 * triangles).  Choices the paper leaves open are stated where they are made.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fno-fast-math -fPIC -shared (see oracle/__init__.py).
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs float arithmetic evaluated in float (FLT_EVAL_METHOD == 0)"
#endif

/* Counter tags: the counter is (pixel or tile, frame, bounce or tag, tag). */
#define TAG_CAMERA 0x43414D45u /* "CAME" */
#define TAG_BSDF 0x42534446u   /* "BSDF" */
#define TAG_INTL 0x494E544Cu   /* "INTL" */
#define TAG_LITE 0x4C495445u   /* "LITE" */

#define MAT_LAMBERT 0u
#define MAT_GGX 1u
#define MAT_MIRROR 2u
#define MAT_DIELECTRIC 4u  /* smooth dielectric: Fresnel reflection or refraction; IOR in the roughness slot */
#define MAT_TRANSLUCENT 5u /* Lambertian transmission into the lower hemisphere */
#define MAT_EMITTER 3u

#define CLS_NONE 0
#define CLS_DIFFUSE 1
#define CLS_GLOSSY 2 /* glossy or specular */
#define DBG_CLS_TRANSLUCENT 3 /* debug output only: a diffuse-class point that transmits */

#define CAT_EMPTY 0
#define CAT_DIFFUSE 1
#define CAT_GLOSSY 2
#define CAT_HYBRID 3

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10, from its definition in Salmon et al. (SC'11): ten rounds of two 32x32
 * multiplications with the round keys bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

static void philox_seed(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                        uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    orc_philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, out);
}

/* 24 high bits of a word as a float in [0, 1). */
static float to_unit(uint32_t x) { return (float)(x >> 8) * 0x1.0p-24f; }

/* ------------------------------------------------------------------------------------ */
/* Sec. 3.3 numbers a tile's pixels in screen order and shuffles the numbers with a linear
 * congruential method whose form it does not give.  Reading: the shuffled number of the
 * tile's i-th pixel is the i-th term of the full-period sequence x_{k+1} = (a x_k + c) mod m. */
void orc_lcg_sequence(uint32_t m, uint32_t a, uint32_t c, uint32_t x0, uint32_t* out) {
    uint64_t x = x0 % m;
    for (uint32_t i = 0; i < m; ++i) {
        out[i] = (uint32_t)x;
        x = ((uint64_t)a * x + c) % m;
    }
}

/* Per tile and per frame parameters (Sec. 3.3: group composition changes from tile to tile
 * and from frame to frame).  With m a power of two, a = 1 (mod 4) and odd c give the full period
 * (Hull-Dobell), so the sequence is a permutation of [0, m). */
void orc_tile_sigma(uint32_t tile_w, uint32_t tile_h, uint32_t tile, uint32_t frame,
                    uint64_t seed, int lcg, uint32_t* sigma, uint32_t* abc_x0) {
    uint32_t m = tile_w * tile_h;
    uint32_t a = 1, c = 1, x0 = 0;
    if (lcg) {
        uint32_t h[4];
        philox_seed(seed, tile, frame, TAG_INTL, 0, h);
        uint32_t q4 = m / 4 > 0 ? m / 4 : 1;
        uint32_t q2 = m / 2 > 0 ? m / 2 : 1;
        a = 4u * (h[0] % q4) + 1u;
        c = 2u * (h[1] % q2) + 1u;
        x0 = h[2] % m;
        orc_lcg_sequence(m, a, c, x0, sigma);
    } else {
        for (uint32_t i = 0; i < m; ++i) sigma[i] = i; /* contiguous groups */
    }
    if (abc_x0) {
        abc_x0[0] = a;
        abc_x0[1] = c;
        abc_x0[2] = x0;
    }
}

/* ------------------------------------------------------------------------------------ */
/* FP32 helpers.  With FLT_EVAL_METHOD == 0 and -ffp-contract=off every operation below is
 * one IEEE round-to-nearest float operation, in the order written. */
typedef struct {
    float x, y, z;
} f3;

static f3 f3m(float x, float y, float z) {
    f3 r = {x, y, z};
    return r;
}
static f3 f3sub(f3 a, f3 b) { return f3m(a.x - b.x, a.y - b.y, a.z - b.z); }
static float f3dot(f3 a, f3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static f3 f3cross(f3 a, f3 b) {
    return f3m(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static f3 f3normalize(f3 a) {
    float l = sqrtf(f3dot(a, a));
    if (l == 0.0f) return f3m(0.0f, 0.0f, 1.0f);
    return f3m(a.x / l, a.y / l, a.z / l);
}

/* sin/cos on [-pi/4, pi/4]: Taylor series to x^11 and x^12 (coefficients 1/n! rounded to
 * float), evaluated by Horner's rule. */
void orc_sincos(float x, float* s, float* c) {
    const float S3 = -0x1.555556p-3f, S5 = 0x1.111112p-7f, S7 = -0x1.a01a02p-13f,
                S9 = 0x1.71de3ap-19f, S11 = -0x1.ae6456p-26f;
    const float C2 = -0x1.0p-1f, C4 = 0x1.555556p-5f, C6 = -0x1.6c16c2p-10f,
                C8 = 0x1.a01a02p-16f, C10 = -0x1.27e4fcp-22f, C12 = 0x1.1eed8ep-29f;
    float x2 = x * x;
    float ps = S11;
    ps = ps * x2 + S9;
    ps = ps * x2 + S7;
    ps = ps * x2 + S5;
    ps = ps * x2 + S3;
    *s = x + (x * x2) * ps;
    float pc = C12;
    pc = pc * x2 + C10;
    pc = pc * x2 + C8;
    pc = pc * x2 + C6;
    pc = pc * x2 + C4;
    pc = pc * x2 + C2;
    *c = 1.0f + x2 * pc;
}

#define PI_D 3.14159265358979323846
#define PI4F 0x1.921fb6p-1f
#define PI2F 0x1.921fb6p+0f
#define INV_SQRT2F 0x1.6a09e6p-1f

/* Cosine-weighted hemisphere sample by the concentric disk map of Shirley and Chiu (1997),
 * lifted to the hemisphere.  The angle is kept in [-pi/4, pi/4] by using the swap identity
 * cos(pi/2 - x) = sin(x) in the second wedge. */
void orc_sample_cosine(float u1, float u2, float* w) {
    float a = 2.0f * u1 - 1.0f;
    float b = 2.0f * u2 - 1.0f;
    float x, y;
    if (a == 0.0f && b == 0.0f) {
        x = 0.0f;
        y = 0.0f;
    } else if (fabsf(a) > fabsf(b)) {
        float s, c;
        orc_sincos(PI4F * (b / a), &s, &c);
        x = a * c;
        y = a * s;
    } else {
        float s, c;
        orc_sincos(PI4F * (a / b), &s, &c);
        x = b * s; /* cos(pi/2 - phi') */
        y = b * c; /* sin(pi/2 - phi') */
    }
    float zz = (1.0f - x * x) - y * y;
    w[0] = x;
    w[1] = y;
    w[2] = sqrtf(zz > 0.0f ? zz : 0.0f);
}

/* cos and sin of 2 pi u for u in [0,1): quadrant q = floor(4u), residual angle in
 * [-pi/4, pi/4) around the quadrant's middle, then the rotation by pi/4 + q pi/2. */
static void sincos_2pi(float u, float* cphi, float* sphi) {
    float t = 4.0f * u;
    int q = (int)t;
    if (q > 3) q = 3;
    float fr = t - (float)q;
    float s, c;
    orc_sincos((fr - 0.5f) * PI2F, &s, &c);
    float c0 = (c - s) * INV_SQRT2F; /* cos(pi/4 + psi) */
    float s0 = (c + s) * INV_SQRT2F; /* sin(pi/4 + psi) */
    switch (q) {
        case 0: *cphi = c0; *sphi = s0; break;
        case 1: *cphi = -s0; *sphi = c0; break;
        case 2: *cphi = -c0; *sphi = -s0; break;
        default: *cphi = s0; *sphi = -c0; break;
    }
}

/* Smith masking for GGX, G1(v) = 2 / (1 + sqrt(1 + alpha^2 tan^2(theta_v))). */
static float ggx_g1(float vz, float a2) {
    float z2 = vz * vz;
    float tan2 = (1.0f - z2) / z2;
    if (tan2 < 0.0f) tan2 = 0.0f;
    return 2.0f / (1.0f + sqrtf(1.0f + a2 * tan2));
}

/* GGX microfacet reflection (Walter et al. 2007): sample m from D(m)(m.n), reflect wo about
 * m.  Weight f cos(wi) / pdf(wi) = F G (wo.m) / (wo.z m.z) with the Schlick Fresnel term
 * (F0 = albedo) and the separable Smith G = G1(wo) G1(wi).  alpha = roughness. */
int orc_sample_ggx(const float* wo, float alpha, const float* f0, float u1, float u2, float* wi,
                   float* weight) {
    float a2 = alpha * alpha;
    float tan2 = (a2 * u1) / (1.0f - u1);
    float cos_t = 1.0f / sqrtf(1.0f + tan2);
    float sin2 = 1.0f - cos_t * cos_t;
    float sin_t = sqrtf(sin2 > 0.0f ? sin2 : 0.0f);
    float cphi, sphi;
    sincos_2pi(u2, &cphi, &sphi);
    f3 m = f3m(sin_t * cphi, sin_t * sphi, cos_t);
    f3 o = f3m(wo[0], wo[1], wo[2]);
    float dot = f3dot(o, m);
    float two_dot = 2.0f * dot;
    f3 r = f3m(two_dot * m.x - o.x, two_dot * m.y - o.y, two_dot * m.z - o.z);
    wi[0] = r.x;
    wi[1] = r.y;
    wi[2] = r.z;
    if (!(o.z > 0.0f) || !(dot > 0.0f) || !(r.z > 0.0f)) {
        weight[0] = weight[1] = weight[2] = 0.0f;
        return 0;
    }
    float g = ggx_g1(o.z, a2) * ggx_g1(r.z, a2);
    float om = 1.0f - dot;
    float om2 = om * om;
    float p5 = (om2 * om2) * om;
    float denom = o.z * m.z;
    for (int k = 0; k < 3; ++k) {
        float F = f0[k] + (1.0f - f0[k]) * p5;
        weight[k] = ((F * g) * dot) / denom;
    }
    return 1;
}

/* GGX reflection BSDF value f(wo, wi) (both in the tangent frame, z up), the density that
 * orc_sample_ggx draws from: f = D(h) G1(wo) G1(wi) F(wo.h) / (4 wo.z wi.z) with the
 * half vector h = normalize(wo + wi), D(h) = alpha^2 / (pi (1 + (alpha^2 - 1) h.z^2)^2)
 * (Walter et al. 2007, Eq. 33), the same Smith G1 and Schlick F.  Zero below either side.
 * Evaluated in double. */
void orc_eval_ggx(const float* wo, const float* wi, float alpha, const float* f0, double* f) {
    f[0] = f[1] = f[2] = 0.0;
    double o[3] = {wo[0], wo[1], wo[2]}, i[3] = {wi[0], wi[1], wi[2]};
    if (!(o[2] > 0.0) || !(i[2] > 0.0)) return;
    double h[3] = {o[0] + i[0], o[1] + i[1], o[2] + i[2]};
    double hl = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (!(hl > 0.0)) return;
    for (int k = 0; k < 3; ++k) h[k] /= hl;
    double a2 = (double)alpha * (double)alpha;
    double q = 1.0 + (a2 - 1.0) * h[2] * h[2];
    double D = a2 / (PI_D * q * q);
    double g = 1.0;
    for (int side = 0; side < 2; ++side) {
        double z = side ? i[2] : o[2];
        double tan2 = (1.0 - z * z) / (z * z);
        if (tan2 < 0.0) tan2 = 0.0;
        g *= 2.0 / (1.0 + sqrt(1.0 + a2 * tan2));
    }
    double oh = o[0] * h[0] + o[1] * h[1] + o[2] * h[2];
    if (!(oh > 0.0)) return;
    double p5 = pow(1.0 - oh, 5.0);
    for (int k = 0; k < 3; ++k) {
        double F = f0[k] + (1.0 - f0[k]) * p5;
        f[k] = D * g * F / (4.0 * o[2] * i[2]);
    }
}

/* Density in solid angle with which orc_sample_ggx draws wi: the microfacet normal h has
 * density D(h) h.z and the reflection maps it with Jacobian 1 / (4 wo.h), so
 * pdf(wi) = D(h) h.z / (4 wo.h), h = normalize(wo + wi); 0 below either side. */
double orc_pdf_ggx(const float* wo, const float* wi, float alpha) {
    double o[3] = {wo[0], wo[1], wo[2]}, i[3] = {wi[0], wi[1], wi[2]};
    if (!(o[2] > 0.0) || !(i[2] > 0.0)) return 0.0;
    double h[3] = {o[0] + i[0], o[1] + i[1], o[2] + i[2]};
    double hl = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (!(hl > 0.0)) return 0.0;
    for (int k = 0; k < 3; ++k) h[k] /= hl;
    double oh = o[0] * h[0] + o[1] * h[1] + o[2] * h[2];
    if (!(oh > 0.0)) return 0.0;
    double a2 = (double)alpha * (double)alpha;
    double q = 1.0 + (a2 - 1.0) * h[2] * h[2];
    double D = a2 / (PI_D * q * q);
    return D * h[2] / (4.0 * oh);
}

/* Orthonormal basis from a unit normal: Duff et al., "Building an Orthonormal Basis,
 * Revisited" (JCGT 2017).  Depends on n only, so coplanar points share a frame. */
static void onb(f3 n, f3* t, f3* b) {
    float sign = copysignf(1.0f, n.z);
    float a = -1.0f / (sign + n.z);
    float bb = (n.x * n.y) * a;
    *t = f3m(1.0f + ((sign * n.x) * n.x) * a, sign * bb, -(sign * n.x));
    *b = f3m(bb, sign + (n.y * n.y) * a, -n.y);
}

void orc_frame(const float* n, float* t, float* b) {
    f3 tt, bb;
    onb(f3m(n[0], n[1], n[2]), &tt, &bb);
    t[0] = tt.x;
    t[1] = tt.y;
    t[2] = tt.z;
    b[0] = bb.x;
    b[1] = bb.y;
    b[2] = bb.z;
}

/* ------------------------------------------------------------------------------------ */
/* Scene and median-split BVH (FP64 bounds). */
typedef struct {
    double lo[3], hi[3];
    int32_t left, right; /* children (inner) */
    int32_t start, count; /* triangle range in order[] (leaf: count > 0) */
} onode;

struct orc_scene {
    uint32_t n_tri, n_mat;
    float* v; /* 9 per triangle */
    uint32_t* tri_mat;
    uint32_t* mat_type;
    float* mat_params; /* 7 per material */
    float env[3];
    onode* nodes;
    uint32_t n_nodes, cap_nodes;
    uint32_t* order;
    double max_abs;
    /* emitter triangles (original ids, ascending) and their cumulative areas */
    uint32_t n_light;
    uint32_t* light_tri;
    float* light_cdf;
    float light_total;
};

static double* g_sort_key; /* qsort has no context argument in C11 */

static int cmp_key(const void* pa, const void* pb) {
    uint32_t a = *(const uint32_t*)pa, b = *(const uint32_t*)pb;
    if (g_sort_key[a] < g_sort_key[b]) return -1;
    if (g_sort_key[a] > g_sort_key[b]) return 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static uint32_t build_node(orc_scene* s, double* cen, uint32_t lo, uint32_t hi) {
    uint32_t id = s->n_nodes++;
    onode* nd = &s->nodes[id];
    for (int k = 0; k < 3; ++k) {
        nd->lo[k] = INFINITY;
        nd->hi[k] = -INFINITY;
    }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = lo; i < hi; ++i) {
        uint32_t t = s->order[i];
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) {
                double x = s->v[9 * t + 3 * v + k];
                if (x < nd->lo[k]) nd->lo[k] = x;
                if (x > nd->hi[k]) nd->hi[k] = x;
            }
        for (int k = 0; k < 3; ++k) {
            if (cen[3 * t + k] < clo[k]) clo[k] = cen[3 * t + k];
            if (cen[3 * t + k] > chi[k]) chi[k] = cen[3 * t + k];
        }
    }
    uint32_t n = hi - lo;
    if (n <= 4) {
        nd->left = nd->right = -1;
        nd->start = (int32_t)lo;
        nd->count = (int32_t)n;
        return id;
    }
    int axis = 0;
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    double* key = (double*)malloc(sizeof(double) * s->n_tri);
    for (uint32_t i = lo; i < hi; ++i) key[s->order[i]] = cen[3 * s->order[i] + axis];
    g_sort_key = key;
    qsort(s->order + lo, n, sizeof(uint32_t), cmp_key);
    free(key);
    uint32_t mid = lo + n / 2;
    nd->start = -1;
    nd->count = 0;
    int32_t l = (int32_t)build_node(s, cen, lo, mid);
    int32_t r = (int32_t)build_node(s, cen, mid, hi);
    s->nodes[id].left = l;
    s->nodes[id].right = r;
    return id;
}

/* Area of a triangle given by 9 floats: half the length of the cross product of two edges,
 * in double. */
double orc_triangle_area(const float* v) {
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = (double)v[3 + k] - (double)v[k];
        e2[k] = (double)v[6 + k] - (double)v[k];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    return 0.5 * sqrt((cx * cx + cy * cy) + cz * cz);
}

orc_scene* orc_scene_new(const float* tri_xyz, uint32_t n_tri, const uint32_t* tri_mat,
                         const uint32_t* mat_type, const float* mat_params, uint32_t n_mat,
                         const float* env) {
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->n_tri = n_tri;
    s->n_mat = n_mat;
    s->v = (float*)malloc(sizeof(float) * 9 * (size_t)n_tri);
    memcpy(s->v, tri_xyz, sizeof(float) * 9 * (size_t)n_tri);
    s->tri_mat = (uint32_t*)malloc(sizeof(uint32_t) * n_tri);
    memcpy(s->tri_mat, tri_mat, sizeof(uint32_t) * n_tri);
    s->mat_type = (uint32_t*)malloc(sizeof(uint32_t) * n_mat);
    memcpy(s->mat_type, mat_type, sizeof(uint32_t) * n_mat);
    s->mat_params = (float*)malloc(sizeof(float) * 7 * n_mat);
    memcpy(s->mat_params, mat_params, sizeof(float) * 7 * n_mat);
    for (int k = 0; k < 3; ++k) s->env[k] = env[k];
    s->max_abs = 0.0;
    for (size_t i = 0; i < 9 * (size_t)n_tri; ++i)
        if (fabs((double)tri_xyz[i]) > s->max_abs) s->max_abs = fabs((double)tri_xyz[i]);
    double* cen = (double*)malloc(sizeof(double) * 3 * n_tri);
    for (uint32_t t = 0; t < n_tri; ++t)
        for (int k = 0; k < 3; ++k)
            cen[3 * t + k] =
                ((double)s->v[9 * t + k] + (double)s->v[9 * t + 3 + k] + (double)s->v[9 * t + 6 + k]) / 3.0;
    s->order = (uint32_t*)malloc(sizeof(uint32_t) * (n_tri ? n_tri : 1));
    for (uint32_t t = 0; t < n_tri; ++t) s->order[t] = t;
    s->cap_nodes = 2 * (n_tri ? n_tri : 1);
    s->nodes = (onode*)malloc(sizeof(onode) * s->cap_nodes);
    s->n_nodes = 0;
    if (n_tri > 0) build_node(s, cen, 0, n_tri);
    free(cen);
    /* Light table for next-event estimation: every emitter triangle in index order, with
     * the running sum of the areas (computed in double from the FP32 vertices) rounded to
     * float.  An emitter is chosen with probability proportional to its area. */
    s->n_light = 0;
    for (uint32_t t = 0; t < n_tri; ++t)
        if (tri_mat[t] < n_mat && mat_type[tri_mat[t]] == MAT_EMITTER) s->n_light++;
    s->light_tri = (uint32_t*)malloc(sizeof(uint32_t) * (s->n_light ? s->n_light : 1));
    s->light_cdf = (float*)malloc(sizeof(float) * (s->n_light ? s->n_light : 1));
    {
        double run = 0.0;
        uint32_t i = 0;
        for (uint32_t t = 0; t < n_tri; ++t) {
            if (!(tri_mat[t] < n_mat && mat_type[tri_mat[t]] == MAT_EMITTER)) continue;
            run += orc_triangle_area(&s->v[9 * t]);
            s->light_tri[i] = t;
            s->light_cdf[i] = (float)run;
            ++i;
        }
        s->light_total = s->n_light ? s->light_cdf[s->n_light - 1] : 0.0f;
    }
    return s;
}

void orc_scene_free(orc_scene* s) {
    if (!s) return;
    free(s->v);
    free(s->tri_mat);
    free(s->mat_type);
    free(s->mat_params);
    free(s->nodes);
    free(s->order);
    free(s->light_tri);
    free(s->light_cdf);
    free(s);
}

uint32_t orc_scene_nodes(const orc_scene* s) { return s->n_nodes; }

/* ------------------------------------------------------------------------------------ */
/* Closest hit in FP64.
 * Hit rule: Moller-Trumbore (1997), t > 0, barycentrics >= 0 (edges inclusive), primitive
 * not the one the ray left.  Closest = smallest t; equal t -> smaller original index.
 * A decision is "fragile" when an FP32 intersector could reasonably decide it differently:
 * another triangle whose hit lies within 1e-6 relative (or eta absolute) of the winner,
 * or a triangle that the ray passes within eta of the boundary of (in the plane normal to
 * the ray) at a depth that could beat the winner, or a candidate at the ray origin.
 * eta = 16 * 2^-24 * (coordinate magnitude + distance), the FP32 rounding scale. */
typedef struct {
    double o[3], d[3];
    double dn[3]; /* unit direction */
    double a1[3], a2[3]; /* orthonormal basis of the plane normal to dn */
    double dlen;
    int32_t skip;
    double eta_ray;
    /* results */
    int32_t best;
    double tbest;
    int found;
    int fragile;
    /* candidates that may beat the winner in FP32 (checked after the search) */
    double threat_tlo[64];
    int n_threat;
    int threat_overflow;
    double hits_t[64];
    int32_t hits_id[64];
    double hits_terr[64]; /* FP32 error scale of t for each hit */
    int hits_edge[64];    /* the ray passes within eta of the hit triangle's boundary */
    int n_hits;
    double terr_best;
} tstate;

static void dsub(const double* a, const double* b, double* r) {
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}
static double ddot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void dcross(const double* a, const double* b, double* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Distance from the 2D origin to segment (a, b) and the segment parameter of the nearest point. */
static double seg_dist2d(const double* a, const double* b, double* lam) {
    double ex = b[0] - a[0], ey = b[1] - a[1];
    double l2 = ex * ex + ey * ey;
    double s = l2 > 0.0 ? -(a[0] * ex + a[1] * ey) / l2 : 0.0;
    if (s < 0.0) s = 0.0;
    if (s > 1.0) s = 1.0;
    *lam = s;
    double px = a[0] + s * ex, py = a[1] + s * ey;
    return sqrt(px * px + py * py);
}

static void test_triangle(const orc_scene* s, uint32_t tri, tstate* st) {
    if ((int32_t)tri == st->skip) return;
    double v0[3], v1[3], v2[3];
    for (int k = 0; k < 3; ++k) {
        v0[k] = s->v[9 * tri + k];
        v1[k] = s->v[9 * tri + 3 + k];
        v2[k] = s->v[9 * tri + 6 + k];
    }
    /* Moller-Trumbore */
    double e1[3], e2[3], pv[3], tv[3], qv[3];
    dsub(v1, v0, e1);
    dsub(v2, v0, e2);
    dcross(st->d, e2, pv);
    double det = ddot(e1, pv);
    int hit = 0;
    double t = 0.0;
    if (det != 0.0) {
        double inv = 1.0 / det;
        dsub(st->o, v0, tv);
        double u = ddot(tv, pv) * inv;
        dcross(tv, e1, qv);
        double v = ddot(st->d, qv) * inv;
        t = ddot(e2, qv) * inv;
        hit = (u >= 0.0 && v >= 0.0 && u + v <= 1.0 && t > 0.0);
    }
    /* Project the triangle onto the plane normal to the ray, with the ray at the origin. */
    const double* V[3] = {v0, v1, v2};
    double q[3][2], along[3], mag = 0.0;
    for (int i = 0; i < 3; ++i) {
        double pmo[3];
        dsub(V[i], st->o, pmo);
        along[i] = ddot(pmo, st->dn);
        q[i][0] = ddot(pmo, st->a1);
        q[i][1] = ddot(pmo, st->a2);
        for (int k = 0; k < 3; ++k)
            if (fabs(pmo[k]) > mag) mag = fabs(pmo[k]);
    }
    double e[3], esum = 0.0;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        e[i] = q[i][0] * q[j][1] - q[i][1] * q[j][0];
        esum += e[i];
    }
    int inside = 1;
    for (int i = 0; i < 3; ++i)
        if (esum >= 0.0 ? e[i] < 0.0 : e[i] > 0.0) inside = 0;
    /* distance from the ray to the projected triangle's boundary and the depth there */
    double dmin = INFINITY, depth_near = 0.0;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        double lam;
        double dist = seg_dist2d(q[i], q[j], &lam);
        if (dist < dmin) {
            dmin = dist;
            depth_near = along[i] + lam * (along[j] - along[i]);
        }
    }
    double eta = 16.0 * 0x1.0p-24 * (st->eta_ray + mag);
    double eta_t = eta / st->dlen;
    int near_edge = dmin < eta;
    /* depth of the part of the triangle the ray passes closest to, in units of t */
    double tau = depth_near / st->dlen;
    if (inside && det != 0.0) tau = t;
    if ((near_edge || inside) && fabs(tau) <= eta_t) st->fragile = 1; /* at the ray origin */
    if (near_edge && tau > -eta_t) {
        if (st->n_threat < 64)
            st->threat_tlo[st->n_threat++] = tau;
        else
            st->threat_overflow = 1;
    }
    if (hit) {
        /* error scale of an FP32 t: coordinate rounding (eta) amplified by the obliquity
         * of the ray to the triangle's plane */
        double nrm[3];
        dcross(e1, e2, nrm);
        double cosv = fabs(ddot(nrm, st->dn)) / sqrt(ddot(nrm, nrm));
        double omag = fabs(st->o[0]);
        if (fabs(st->o[1]) > omag) omag = fabs(st->o[1]);
        if (fabs(st->o[2]) > omag) omag = fabs(st->o[2]);
        double terr = 4.0 * 0x1.0p-24 * (mag + omag) / st->dlen / (cosv > 1e-12 ? cosv : 1e-12);
        if (st->n_hits < 64) {
            st->hits_t[st->n_hits] = t;
            st->hits_id[st->n_hits] = (int32_t)tri;
            st->hits_terr[st->n_hits] = terr;
            st->hits_edge[st->n_hits] = near_edge;
            st->n_hits++;
        } else {
            st->fragile = 1;
        }
        if (!st->found || t < st->tbest || (t == st->tbest && (int32_t)tri < st->best)) {
            st->found = 1;
            st->tbest = t;
            st->best = (int32_t)tri;
            st->terr_best = terr;
        }
    }
}

static void dnorm3(double* a) {
    double l = sqrt(ddot(a, a));
    a[0] /= l;
    a[1] /= l;
    a[2] /= l;
}

static int box_hit(const onode* nd, const tstate* st, double pad, double tcull) {
    double tn = -2.0 * pad / st->dlen, tf = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double lo = nd->lo[k] - pad, hi = nd->hi[k] + pad;
        if (st->d[k] == 0.0) {
            if (st->o[k] < lo || st->o[k] > hi) return 0;
            continue;
        }
        double t0 = (lo - st->o[k]) / st->d[k];
        double t1 = (hi - st->o[k]) / st->d[k];
        if (t0 > t1) {
            double x = t0;
            t0 = t1;
            t1 = x;
        }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
    }
    tf *= 1.0 + 1e-12;
    return tn <= tf && tn <= tcull;
}

/* Closest-hit search; leaves the hits, the near-edge candidates and the winner in st. */
static void traverse(const orc_scene* s, const double* o, const double* d, int32_t skip, int use_bvh, tstate* stp,
                     double* omax_out) {
    tstate st;
    memset(&st, 0, sizeof(st));
    for (int k = 0; k < 3; ++k) {
        st.o[k] = o[k];
        st.d[k] = d[k];
    }
    st.dlen = sqrt(ddot(d, d));
    for (int k = 0; k < 3; ++k) st.dn[k] = d[k] / st.dlen;
    {
        double ax[3] = {0.0, 0.0, 0.0};
        int kmin = 0;
        for (int k = 1; k < 3; ++k)
            if (fabs(st.dn[k]) < fabs(st.dn[kmin])) kmin = k;
        ax[kmin] = 1.0;
        dcross(st.dn, ax, st.a1);
        dnorm3(st.a1);
        dcross(st.dn, st.a1, st.a2);
    }
    st.skip = skip;
    double omax = fabs(o[0]);
    if (fabs(o[1]) > omax) omax = fabs(o[1]);
    if (fabs(o[2]) > omax) omax = fabs(o[2]);
    st.eta_ray = omax > s->max_abs ? omax : s->max_abs;
    st.best = -1;
    if (!use_bvh || s->n_nodes == 0) {
        for (uint32_t t = 0; t < s->n_tri; ++t) test_triangle(s, t, &st);
    } else {
        /* pad boxes by the largest eta any triangle of this ray can have */
        double pad = 16.0 * 0x1.0p-24 * (4.0 * (omax + s->max_abs));
        uint32_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const onode* nd = &s->nodes[stack[--sp]];
            double tcull = st.found ? st.tbest * (1.0 + 1e-5) + 2.0 * pad / st.dlen : INFINITY;
            if (!box_hit(nd, &st, pad, tcull)) continue;
            if (nd->count > 0) {
                for (int32_t i = 0; i < nd->count; ++i) test_triangle(s, s->order[nd->start + i], &st);
            } else {
                stack[sp++] = (uint32_t)nd->left;
                stack[sp++] = (uint32_t)nd->right;
            }
        }
    }
    *stp = st;
    *omax_out = omax;
}

static void trace_ray_bound(const orc_scene* s, const double* o, const double* d, int32_t skip, int use_bvh,
                            int32_t* prim, double* tout, uint8_t* fragile, double* terr) {
    tstate st;
    double omax;
    traverse(s, o, d, skip, use_bvh, &st, &omax);
    if (st.found) {
        double eta_t = 16.0 * 0x1.0p-24 * (2.0 * (omax + s->max_abs)) / st.dlen;
        double band = st.tbest * 1e-6 + eta_t;
        for (int i = 0; i < st.n_hits; ++i)
            if (st.hits_id[i] != st.best && st.hits_t[i] - st.tbest <= band) st.fragile = 1;
        for (int i = 0; i < st.n_threat; ++i)
            if (st.threat_tlo[i] <= st.tbest + band) st.fragile = 1;
    } else if (st.n_threat > 0) {
        st.fragile = 1;
    }
    if (st.threat_overflow) st.fragile = 1;
    *prim = st.found ? st.best : -1;
    *tout = st.found ? st.tbest : INFINITY;
    /* bit 0: the hit/miss or primitive decision is fragile; bit 1: t itself is
     * ill-conditioned in FP32 (error scale above 1e-5 t: oblique hits, hits close to the
     * ray origin relative to the coordinates' magnitude) */
    int tbad = st.found && st.terr_best > 1e-5 * st.tbest;
    *fragile = (uint8_t)((st.fragile ? 1 : 0) | (tbad ? 2 : 0));
    if (terr) *terr = st.found ? st.terr_best : 0.0;
}

static void trace_ray(const orc_scene* s, const double* o, const double* d, int32_t skip, int use_bvh,
                      int32_t* prim, double* tout, uint8_t* fragile) {
    trace_ray_bound(s, o, d, skip, use_bvh, prim, tout, fragile, NULL);
}

/* Visibility of a shadow ray: occluded when some triangle other than `skip` is hit at
 * 0 < t < tmax (t in units of d).  Fragile when an FP32 traversal could decide differently:
 * unless a hit well before tmax (by the band below) on a triangle whose boundary the ray
 * does not graze settles it, any grazed triangle in front of tmax, any hit within the band
 * of tmax, or a candidate at the ray origin makes the answer fragile. */
static void shadow_ray(const orc_scene* s, const double* o, const double* d, double tmax, int32_t skip,
                       int use_bvh, int* occluded, int* fragile) {
    tstate st;
    double omax;
    traverse(s, o, d, skip, use_bvh, &st, &omax);
    double eta_t = 16.0 * 0x1.0p-24 * (2.0 * (omax + s->max_abs)) / st.dlen;
    double band = tmax * 1e-6 + eta_t;
    *occluded = st.found && st.tbest < tmax;
    int robust = 0;
    for (int i = 0; i < st.n_hits; ++i)
        if (st.hits_t[i] < tmax - band && !st.hits_edge[i]) robust = 1;
    int fr = 0;
    if (!robust) {
        for (int i = 0; i < st.n_hits; ++i)
            if (st.hits_t[i] <= tmax + band) fr = 1;
        for (int i = 0; i < st.n_threat; ++i)
            if (st.threat_tlo[i] < tmax + band) fr = 1;
        if (st.fragile || st.threat_overflow || st.n_hits >= 64) fr = 1;
    }
    *fragile = fr;
}

void orc_shadow(const orc_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n, int use_bvh,
                uint8_t* occluded, uint8_t* fragile) {
    for (uint32_t i = 0; i < n; ++i) {
        double o[3] = {rays[8 * i + 0], rays[8 * i + 1], rays[8 * i + 2]};
        double d[3] = {rays[8 * i + 4], rays[8 * i + 5], rays[8 * i + 6]};
        int oc, fr;
        shadow_ray(s, o, d, (double)rays[8 * i + 7], skip_prim ? skip_prim[i] : -1, use_bvh, &oc, &fr);
        occluded[i] = (uint8_t)oc;
        fragile[i] = (uint8_t)fr;
    }
}

/* Light sample for next-event estimation from three uniforms in [0, 1).
 * Emitter choice: x = u0 * total (float); the first emitter whose running area exceeds x
 * (the last one if rounding leaves none), i.e. probability area / total.
 * Point: uniform on the triangle by the square-root map (Shirley & Chiu / Turk 1990):
 * with s = sqrt(u1), p = (1 - s) v0 + s (1 - u2) v1 + s u2 v2, in float.
 * Returns the emitter's original triangle index, -1 if the scene has no emitter. */
int32_t orc_light_sample(const orc_scene* s, float u0, float u1, float u2, float* p) {
    if (s->n_light == 0) return -1;
    float x = u0 * s->light_total;
    uint32_t i = 0;
    while (i < s->n_light && !(x < s->light_cdf[i])) ++i;
    if (i == s->n_light) i = s->n_light - 1;
    const uint32_t t = s->light_tri[i];
    const float* v = &s->v[9 * t];
    float sq = sqrtf(u1);
    float b0 = 1.0f - sq, b1 = sq * (1.0f - u2), b2 = sq * u2;
    for (int k = 0; k < 3; ++k) p[k] = (v[k] * b0 + v[3 + k] * b1) + v[6 + k] * b2;
    return (int32_t)t;
}

uint32_t orc_scene_lights(const orc_scene* s, float* total) {
    if (total) *total = s->light_total;
    return s->n_light;
}

void orc_trace(const orc_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n, int use_bvh,
               int32_t* prim, double* t, uint8_t* fragile) {
    orc_trace_bound(s, rays, skip_prim, n, use_bvh, prim, t, fragile, NULL);
}

void orc_trace_bound(const orc_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n, int use_bvh,
                     int32_t* prim, double* t, uint8_t* fragile, double* terr) {
    for (uint32_t i = 0; i < n; ++i) {
        double o[3] = {rays[8 * i + 0], rays[8 * i + 1], rays[8 * i + 2]};
        double d[3] = {rays[8 * i + 4], rays[8 * i + 5], rays[8 * i + 6]};
        trace_ray_bound(s, o, d, skip_prim ? skip_prim[i] : -1, use_bvh, &prim[i], &t[i], &fragile[i],
                        terr ? &terr[i] : NULL);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Camera: pinhole, vertical field of view; basis in double rounded once to float. */
typedef struct {
    f3 pos, fwd, right, up;
    float tx, ty; /* tan(vfov/2) * aspect, tan(vfov/2) */
} cam_basis;

static void dnorm(double* a) {
    double l = sqrt(ddot(a, a));
    a[0] /= l;
    a[1] /= l;
    a[2] /= l;
}

static cam_basis make_camera(const orc_camera* c) {
    double p[3] = {c->pos[0], c->pos[1], c->pos[2]};
    double la[3] = {c->look_at[0], c->look_at[1], c->look_at[2]};
    double up[3] = {c->up[0], c->up[1], c->up[2]};
    double f[3], r[3], u[3];
    dsub(la, p, f);
    dnorm(f);
    dcross(f, up, r);
    dnorm(r);
    dcross(r, f, u);
    double th = tan(c->vfov_deg * (3.14159265358979323846 / 180.0) * 0.5);
    cam_basis b;
    b.pos = f3m(c->pos[0], c->pos[1], c->pos[2]);
    b.fwd = f3m((float)f[0], (float)f[1], (float)f[2]);
    b.right = f3m((float)r[0], (float)r[1], (float)r[2]);
    b.up = f3m((float)u[0], (float)u[1], (float)u[2]);
    b.ty = (float)th;
    b.tx = (float)(th * ((double)c->width / (double)c->height));
    return b;
}

/* Primary ray through pixel (px, py) jittered by (u, v). */
static f3 camera_dir(const cam_basis* b, uint32_t w, uint32_t h, uint32_t px, uint32_t py, float u,
                     float v) {
    float sx = ((2.0f * ((float)px + u)) / (float)w - 1.0f) * b->tx;
    float sy = (1.0f - (2.0f * ((float)py + v)) / (float)h) * b->ty;
    f3 d = f3m((b->fwd.x + sx * b->right.x) + sy * b->up.x, (b->fwd.y + sx * b->right.y) + sy * b->up.y,
               (b->fwd.z + sx * b->right.z) + sy * b->up.z);
    return f3normalize(d);
}

void orc_camera_ray(const orc_camera* cam, uint32_t px, uint32_t py, float u, float v, float* d) {
    cam_basis b = make_camera(cam);
    f3 r = camera_dir(&b, cam->width, cam->height, px, py, u, v);
    d[0] = r.x;
    d[1] = r.y;
    d[2] = r.z;
}

/* ------------------------------------------------------------------------------------ */
/* Path state of one slot of a tile. */
typedef struct {
    int32_t pixel; /* -1: slot of a pixel outside the image */
    int alive;
    int taint;
    int staint;    /* a fragile shadow-ray decision of this pixel (does not spread to its group) */
    double pdf;    /* solid-angle density of the direction just traced (0: camera ray or mirror) */
    float beta[3];
    double L[3];
    double o[3];
    f3 d;
    int32_t hit; /* original triangle index of the last trace, -1 miss */
    double t;
    /* shading point */
    f3 n, T, B, wo;
    int cls;
    int cosgl;   /* a GGX point in the diffuse class while reusing: cosine sampling, pi f weights */
    uint32_t mat;
    /* direction chosen at this step */
    f3 wl;
    float w[3];
    int valid;
    float hemi;  /* +1: the diffuse lobe is the upper hemisphere, -1: the lower (translucent) */
    int front;   /* the incoming ray met the triangle's front face (cross(v1-v0, v2-v0) side) */
} pstate;

static void shade_setup(const orc_scene* s, pstate* ps, float diffuse_roughness, int reuse_now) {
    const float* v = &s->v[9 * ps->hit];
    f3 v0 = f3m(v[0], v[1], v[2]), v1 = f3m(v[3], v[4], v[5]), v2 = f3m(v[6], v[7], v[8]);
    f3 ng = f3normalize(f3cross(f3sub(v1, v0), f3sub(v2, v0)));
    /* two-sided: the shading normal faces the incoming ray */
    ps->front = f3dot(ng, ps->d) < 0.0f;
    f3 n = ps->front ? ng : f3m(-ng.x, -ng.y, -ng.z);
    ps->n = n;
    onb(n, &ps->T, &ps->B);
    f3 md = f3m(-ps->d.x, -ps->d.y, -ps->d.z);
    ps->wo = f3m(f3dot(md, ps->T), f3dot(md, ps->B), f3dot(md, n));
    ps->mat = s->tri_mat[ps->hit];
    uint32_t ty = s->mat_type[ps->mat];
    /* Transmission (the paper's future work, Sec. 6): a Lambertian transmitter joins the
     * diffuse class with its lobe in the lower hemisphere; a smooth dielectric is specular. */
    ps->cls = (ty == MAT_LAMBERT || ty == MAT_TRANSLUCENT) ? CLS_DIFFUSE : CLS_GLOSSY;
    /* roughness threshold of the classes: a rough GGX point joins the diffuse class */
    const int rough = ty == MAT_GGX && diffuse_roughness > 0.0f &&
                      s->mat_params[7 * ps->mat + 3] >= diffuse_roughness;
    if (rough) ps->cls = CLS_DIFFUSE;
    ps->cosgl = rough && reuse_now;
    ps->hemi = ty == MAT_TRANSLUCENT ? -1.0f : 1.0f;
}

/* Weight pi f(wo, wi) (= f cos / p_cos) of a cosine-class GGX point for the tangent-space
 * direction wl; the direction is usable when both it and wo lie above the surface. */
static void rough_weight(const orc_scene* s, pstate* ps, f3 wl) {
    const float* mp = &s->mat_params[7 * ps->mat];
    float wo[3] = {ps->wo.x, ps->wo.y, ps->wo.z}, wi[3] = {wl.x, wl.y, wl.z};
    double f[3];
    orc_eval_ggx(wo, wi, mp[3], mp, f);
    for (int k = 0; k < 3; ++k) ps->w[k] = (float)(PI_D * f[k]);
    ps->valid = wl.z > 0.0f && ps->wo.z > 0.0f;
}

/* Smooth dielectric (IOR eta inside, 1 outside; the inside lies behind the front face):
 * unpolarised Fresnel reflectance F from the relative index e = eta_i / eta_t, reflection
 * when u < F (total internal reflection when sin^2 t >= 1), else refraction by Snell's law,
 * wi = (-e wo.x, -e wo.y, -cos t).  Both branches carry the tint (F and 1 - F cancel
 * against their selection probabilities).  FP32, one fixed operation order. */
int orc_sample_dielectric(const float* wo, float eta, int front, float u, float* wi) {
    float eta_i = front ? 1.0f : eta, eta_t = front ? eta : 1.0f;
    float e = eta_i / eta_t;
    float ci = wo[2];
    float s2 = (e * e) * (1.0f - ci * ci);
    float F = 1.0f, ct = 0.0f;
    if (s2 < 1.0f) {
        ct = sqrtf(1.0f - s2);
        float rs = (eta_i * ci - eta_t * ct) / (eta_i * ci + eta_t * ct);
        float rp = (eta_t * ci - eta_i * ct) / (eta_t * ci + eta_i * ct);
        F = 0.5f * (rs * rs + rp * rp);
    }
    if (u < F) {
        wi[0] = -wo[0];
        wi[1] = -wo[1];
        wi[2] = wo[2];
        return 0;
    }
    wi[0] = -(e * wo[0]);
    wi[1] = -(e * wo[1]);
    wi[2] = -ct;
    return 1;
}

static void bsdf_rand(uint64_t seed, const pstate* ps, uint32_t frame, uint32_t bounce, float* u1, float* u2) {
    uint32_t h[4];
    philox_seed(seed, (uint32_t)ps->pixel, frame, bounce, TAG_BSDF, h);
    *u1 = to_unit(h[0]);
    *u2 = to_unit(h[1]);
}

/* The member's own BSDF sample (the independent / glossy-group rule). */
static void own_sample(const orc_scene* s, uint64_t seed, uint32_t frame, uint32_t bounce, pstate* ps) {
    float u1, u2, wl[3];
    bsdf_rand(seed, ps, frame, bounce, &u1, &u2);
    const float* mp = &s->mat_params[7 * ps->mat];
    uint32_t ty = s->mat_type[ps->mat];
    if (ty == MAT_LAMBERT) {
        orc_sample_cosine(u1, u2, wl);
        ps->wl = f3m(wl[0], wl[1], wl[2]);
        for (int k = 0; k < 3; ++k) ps->w[k] = mp[k];
        ps->valid = 1;
    } else if (ps->cosgl) { /* a GGX point of the diffuse class: cosine sample, pi f weight */
        orc_sample_cosine(u1, u2, wl);
        ps->wl = f3m(wl[0], wl[1], wl[2]);
        rough_weight(s, ps, ps->wl);
    } else if (ty == MAT_GGX) {
        float wo[3] = {ps->wo.x, ps->wo.y, ps->wo.z};
        ps->valid = orc_sample_ggx(wo, mp[3], mp, u1, u2, wl, ps->w);
        ps->wl = f3m(wl[0], wl[1], wl[2]);
    } else if (ty == MAT_TRANSLUCENT) {
        orc_sample_cosine(u1, u2, wl);
        ps->wl = f3m(wl[0], wl[1], -wl[2]);
        for (int k = 0; k < 3; ++k) ps->w[k] = mp[k];
        ps->valid = 1;
    } else if (ty == MAT_DIELECTRIC) {
        float wo[3] = {ps->wo.x, ps->wo.y, ps->wo.z};
        orc_sample_dielectric(wo, mp[3], ps->front, u1, wl);
        ps->wl = f3m(wl[0], wl[1], wl[2]);
        for (int k = 0; k < 3; ++k) ps->w[k] = mp[k];
        ps->valid = ps->wo.z > 0.0f;
    } else { /* mirror */
        ps->wl = f3m(-ps->wo.x, -ps->wo.y, ps->wo.z);
        for (int k = 0; k < 3; ++k) ps->w[k] = mp[k];
        ps->valid = ps->wo.z > 0.0f;
    }
}

static void take_direction(const orc_scene* s, pstate* ps, f3 wl) {
    const float* mp = &s->mat_params[7 * ps->mat];
    ps->wl = wl;
    if (ps->cosgl) {
        rough_weight(s, ps, wl);
        return;
    }
    for (int k = 0; k < 3; ++k) ps->w[k] = mp[k]; /* Lambert: f cos / p_cos = albedo */
    ps->valid = 1;
}

/* A shared tangent-space direction taken into the member's own diffuse lobe: its normal
 * component becomes hemi * |z| (a translucent member mirrors it through the tangent plane),
 * so a cosine-distributed direction stays cosine-distributed in either lobe. */
static f3 into_lobe(const pstate* ps, f3 wl) { return f3m(wl.x, wl.y, ps->hemi * fabsf(wl.z)); }

static f3 to_world(const pstate* ps, f3 l) {
    return f3m((ps->T.x * l.x + ps->B.x * l.y) + ps->n.x * l.z, (ps->T.y * l.x + ps->B.y * l.y) + ps->n.y * l.z,
               (ps->T.z * l.x + ps->B.z * l.y) + ps->n.z * l.z);
}

/* Pairwise tree sum over the K slots of a group: level l adds slots j and j + 2^l. */
static f3 tree_sum(f3* v, uint32_t k) {
    for (uint32_t stride = 1; stride < k; stride *= 2)
        for (uint32_t j = 0; j + stride < k; j += 2 * stride)
            v[j] = f3m(v[j].x + v[j + stride].x, v[j].y + v[j + stride].y, v[j].z + v[j + stride].z);
    return v[0];
}

/* Solid-angle density with which the shading point's own BSDF sampling draws the
 * tangent-space direction wl: cos / pi (Lambert), the GGX reflection density (GGX), 0 for
 * the mirror's delta distribution (its emission is never weighed). */
static double bsdf_pdf(const orc_scene* s, const pstate* ps, f3 wl) {
    uint32_t ty = s->mat_type[ps->mat];
    if (ty == MAT_LAMBERT) return wl.z > 0.0f ? (double)wl.z / PI_D : 0.0;
    if (ty == MAT_TRANSLUCENT) return wl.z < 0.0f ? -(double)wl.z / PI_D : 0.0;
    if (ps->cosgl) return wl.z > 0.0f ? (double)wl.z / PI_D : 0.0;
    if (ty == MAT_GGX) {
        float wo[3] = {ps->wo.x, ps->wo.y, ps->wo.z}, wi[3] = {wl.x, wl.y, wl.z};
        return orc_pdf_ggx(wo, wi, s->mat_params[7 * ps->mat + 3]);
    }
    return 0.0;
}

/* MIS weight of emission met by the path's last trace (power heuristic): the ray's
 * direction had density ps->pdf (0: camera ray or mirror, weight 1); a light sample would
 * have reached the same point with density r^2 / (cos_l A). */
static double emit_weight(const orc_scene* s, const pstate* ps) {
    if (ps->pdf == 0.0) return 1.0;
    const float* lv = &s->v[9 * ps->hit];
    double e1[3], e2[3], nl[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = (double)lv[3 + k] - (double)lv[k];
        e2[k] = (double)lv[6 + k] - (double)lv[k];
    }
    dcross(e1, e2, nl);
    double d[3] = {ps->d.x, ps->d.y, ps->d.z};
    double dd = ddot(d, d);
    double cos_l = fabs(ddot(nl, d)) / sqrt(ddot(nl, nl) * dd);
    if (!(cos_l > 0.0)) return 1.0;
    double p_l = ps->t * ps->t * dd / (cos_l * (double)s->light_total);
    return ps->pdf * ps->pdf / (ps->pdf * ps->pdf + p_l * p_l);
}

/* Spawn point of the next ray: p = o + t d in FP64, offset by 2^-18 max(1, |p|_inf) along
 * the shading normal times side (+1 for a ray leaving on the incoming side, -1 for a
 * transmitted one), so that the new ray clears the surface it leaves. */
void orc_spawn_point(const double* o, const float* d, double t, const float* n, double side, double* out) {
    double pt[3], amax = 1.0;
    for (int k = 0; k < 3; ++k) {
        pt[k] = o[k] + t * (double)d[k];
        if (fabs(pt[k]) > amax) amax = fabs(pt[k]);
    }
    double eps = 0x1.0p-18 * amax;
    for (int k = 0; k < 3; ++k) out[k] = pt[k] + (side * eps) * (double)n[k];
}

static void spawn_point(const pstate* ps, double side, double* out) {
    float d[3] = {ps->d.x, ps->d.y, ps->d.z}, n[3] = {ps->n.x, ps->n.y, ps->n.z};
    orc_spawn_point(ps->o, d, ps->t, n, side, out);
}

#define SHADOW_TMAX (1.0 - 0x1.0p-10) /* shadow rays run to 1 - 2^-10 of the way to the light point */
#define NEE_COS_FRAGILE 1e-4

/* Next-event estimation at a non-specular shading point (a standard estimator; the paper
 * is silent): one emitter point drawn by area, p_A = 1 / total emitter area A, and
 *   L += w_l beta f(wo, wi) Le cos_i cos_l / r^2 / p_A   if the shadow ray reaches it,
 * with wi toward the point, cos_i at the shading point, cos_l at the (two-sided) emitter.
 * The same emission can also be met by the path's next BSDF-sampled ray; the two
 * estimates are combined by multiple importance sampling with the power heuristic (Veach
 * & Guibas 1995): in solid angle the light sample has density p_l = r^2 / (cos_l A) and the
 * BSDF density p_b is the shading point's own (bsdf_pdf); w_l = p_l^2 / (p_l^2 + p_b^2),
 * and an emitter hit by the BSDF-sampled ray weighs its emission by the complement
 * (emit_weight).  Both weights use the same two densities, so the estimate keeps the
 * mean of plain path tracing whenever the continuation direction has density p_b. */
static void next_event(const orc_scene* s, uint64_t seed, uint32_t frame, uint32_t bounce, pstate* ps,
                       int32_t light_pixel, uint64_t* counters) {
    uint32_t h[4];
    philox_seed(seed, (uint32_t)light_pixel, frame, bounce, TAG_LITE, h);
    float pl[3];
    int32_t lt = orc_light_sample(s, to_unit(h[0]), to_unit(h[1]), to_unit(h[2]), pl);
    if (lt < 0) return;
    double o[3], dl[3];
    spawn_point(ps, (double)ps->hemi, o);
    for (int k = 0; k < 3; ++k) dl[k] = (double)pl[k] - o[k];
    double r2 = ddot(dl, dl);
    if (!(r2 > 0.0)) return;
    double r = sqrt(r2);
    double nn[3] = {ps->n.x, ps->n.y, ps->n.z};
    double cos_i = (double)ps->hemi * ddot(nn, dl) / r; /* on the lobe's side of the surface */
    const float* lv = &s->v[9 * lt];
    double e1[3], e2[3], nl[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = (double)lv[3 + k] - (double)lv[k];
        e2[k] = (double)lv[6 + k] - (double)lv[k];
    }
    dcross(e1, e2, nl);
    double cos_l = fabs(ddot(nl, dl)) / (sqrt(ddot(nl, nl)) * r);
    if (fabs(cos_i) < NEE_COS_FRAGILE || cos_l < NEE_COS_FRAGILE) ps->staint = 1;
    if (!(cos_i > 0.0) || !(cos_l > 0.0)) return;
    int occluded, fragile;
    shadow_ray(s, o, dl, SHADOW_TMAX, ps->hit, 1, &occluded, &fragile);
    counters[3]++;
    if (fragile) {
        ps->staint = 1;
        counters[4]++;
    }
    if (occluded) return;
    const float* mp = &s->mat_params[7 * ps->mat];
    const float* le = &s->mat_params[7 * s->tri_mat[lt] + 4];
    /* the light direction in the shading frame */
    double wi[3] = {dl[0] / r, dl[1] / r, dl[2] / r};
    double T[3] = {ps->T.x, ps->T.y, ps->T.z}, B[3] = {ps->B.x, ps->B.y, ps->B.z};
    f3 wil = f3m((float)ddot(T, wi), (float)ddot(B, wi), (float)ddot(nn, wi));
    double f[3];
    if (s->mat_type[ps->mat] == MAT_LAMBERT || s->mat_type[ps->mat] == MAT_TRANSLUCENT) {
        for (int k = 0; k < 3; ++k) f[k] = (double)mp[k] / PI_D;
    } else {
        float wo[3] = {ps->wo.x, ps->wo.y, ps->wo.z}, wv[3] = {wil.x, wil.y, wil.z};
        orc_eval_ggx(wo, wv, mp[3], mp, f);
    }
    double p_l = r2 / (cos_l * (double)s->light_total);
    double p_b = bsdf_pdf(s, ps, wil);
    double wl = p_l * p_l / (p_l * p_l + p_b * p_b);
    double g = cos_i * cos_l / r2 * (double)s->light_total * wl;
    for (int k = 0; k < 3; ++k) ps->L[k] += (double)ps->beta[k] * f[k] * (double)le[k] * g;
}

/* Replay capture of trace row di: the ray as a float record, its throughput and density. */
static void capture_ray(const pstate* ps, orc_outputs* out, uint32_t di) {
    if (!out->dbg_ray) return;
    float* r = &out->dbg_ray[8 * (size_t)di];
    int32_t skip = ps->hit;
    r[0] = (float)ps->o[0];
    r[1] = (float)ps->o[1];
    r[2] = (float)ps->o[2];
    memcpy(&r[3], &skip, sizeof(skip));
    r[4] = ps->d.x;
    r[5] = ps->d.y;
    r[6] = ps->d.z;
    r[7] = INFINITY;
    for (int k = 0; k < 3; ++k) out->dbg_beta[4 * (size_t)di + k] = ps->beta[k];
    out->dbg_beta[4 * (size_t)di + 3] = (float)ps->pdf;
}

static void trace_path(const orc_scene* s, pstate* ps, uint64_t* counters) {
    int32_t prim;
    double t;
    uint8_t fr;
    double d[3] = {ps->d.x, ps->d.y, ps->d.z};
    trace_ray(s, ps->o, d, ps->hit, 1, &prim, &t, &fr);
    ps->hit = prim;
    ps->t = t;
    if (fr & 1) {
        ps->taint = 1;
        counters[2]++;
    }
}

/* One shading step of the path (bounce b, Sec. 3.2) over the m slots of one tile, in the
 * paper's order: the hits of trace b-1 are shaded (environment, emission, or a shading point
 * with its frame and class), next-event estimation adds its light samples, then every group
 * is classified and its members' exit directions are chosen (own samples, or the reused
 * direction of the group's category), and each continuing path spawns its next ray and
 * multiplies its throughput.  The per-pixel debug outputs, when requested, go to row
 * dbg_row of out's per-bounce arrays. */
static void shade_step(const orc_scene* s, const orc_params* p, uint32_t f, uint32_t b, uint32_t m, pstate* slot,
                       f3* sumbuf, orc_outputs* out, uint32_t dbg_row, uint64_t* cnt_local) {
    const uint32_t K = p->k;
    /* shade the hits of trace b-1: environment, emission, or a shading point */
    for (uint32_t j = 0; j < m; ++j) {
        pstate* ps = &slot[j];
        if (ps->pixel < 0 || !ps->alive) continue;
        if (ps->hit < 0) {
            for (int k = 0; k < 3; ++k) ps->L[k] += (double)(ps->beta[k] * s->env[k]);
            ps->alive = 0;
            continue;
        }
        uint32_t mt = s->mat_type[s->tri_mat[ps->hit]];
        if (mt == MAT_EMITTER) {
            const float* mp = &s->mat_params[7 * s->tri_mat[ps->hit]];
            double wb = (p->opts & ORC_OPT_NEE) ? emit_weight(s, ps) : 1.0;
            for (int k = 0; k < 3; ++k) ps->L[k] += (double)(ps->beta[k] * mp[4 + k]) * wb;
            ps->alive = 0;
            continue;
        }
        shade_setup(s, ps, p->diffuse_roughness,
                    (p->mode == ORC_DIRECTION_REUSE || p->mode == ORC_WORLD_REUSE) &&
                        (p->reuse_depth == 0 || b <= p->reuse_depth));
    }
    /* next-event estimation at the shading points; with shared light samples
     * every member of a group joins the point drawn from the stream of the
     * group's first alive member (each member's point is still distributed by
     * area, so every pixel's estimate keeps its mean) */
    if (p->opts & ORC_OPT_NEE) {
        for (uint32_t g = 0; g < m / K; ++g) {
            pstate* G = &slot[g * K];
            int32_t owner = -1;
            for (uint32_t j = 0; j < K && owner < 0; ++j)
                if (G[j].pixel >= 0 && G[j].alive) owner = G[j].pixel;
            for (uint32_t j = 0; j < K; ++j) {
                pstate* ps = &G[j];
                if (ps->pixel < 0 || !ps->alive) continue;
                uint32_t ty = s->mat_type[ps->mat];
                if (ty == MAT_MIRROR || ty == MAT_DIELECTRIC) continue;
                next_event(s, p->seed, f, b, ps, (p->opts & ORC_OPT_NEE_SHARED) ? owner : ps->pixel,
                           cnt_local);
            }
        }
    }
    const int reuse_now = (p->mode == ORC_DIRECTION_REUSE || p->mode == ORC_WORLD_REUSE) &&
                          (p->reuse_depth == 0 || b <= p->reuse_depth);
    for (uint32_t g = 0; g < m / K; ++g) {
        pstate* G = &slot[g * K];
        /* Sec. 3.2: classify the group by the materials of its shading points */
        int nd = 0, ng = 0, taint = 0;
        for (uint32_t j = 0; j < K; ++j) {
            if (G[j].pixel < 0) continue;
            taint |= G[j].taint;
            if (!G[j].alive) continue;
            if (G[j].cls == CLS_DIFFUSE) nd++;
            else ng++;
        }
        int cat = nd && ng ? CAT_HYBRID : (nd ? CAT_DIFFUSE : (ng ? CAT_GLOSSY : CAT_EMPTY));
        if (reuse_now && taint)
            for (uint32_t j = 0; j < K; ++j)
                if (G[j].pixel >= 0) G[j].taint = 1;
        for (uint32_t j = 0; j < K; ++j)
            if (G[j].pixel >= 0 && G[j].alive) own_sample(s, p->seed, f, b, &G[j]);
        if (reuse_now && p->mode == ORC_WORLD_REUSE) {
            /* Sec. 3.1 direct reuse: the first member's world-space exit direction,
             * each member weighing it with its own material */
            int donor = -1;
            for (uint32_t j = 0; j < K && donor < 0; ++j)
                if (G[j].pixel >= 0 && G[j].alive) donor = (int)j;
            if (donor >= 0 && G[donor].valid) {
                f3 wd = to_world(&G[donor], G[donor].wl);
                for (uint32_t j = 0; j < K; ++j) {
                    pstate* ps = &G[j];
                    if (ps->pixel < 0 || !ps->alive || ps->cls != CLS_DIFFUSE) continue;
                    f3 l = f3m(f3dot(wd, ps->T), f3dot(wd, ps->B), f3dot(wd, ps->n));
                    take_direction(s, ps, l);
                    if (!(ps->hemi * l.z > 0.0f)) ps->valid = 0; /* outside the lobe: f = 0 */
                }
            }
        } else if (reuse_now && cat == CAT_DIFFUSE) {
            /* diffuse group: every member reuses the first member's exit direction */
            int donor = -1;
            for (uint32_t j = 0; j < K && donor < 0; ++j)
                if (G[j].pixel >= 0 && G[j].alive) donor = (int)j;
            f3 wl = G[donor].wl;
            for (uint32_t j = 0; j < K; ++j)
                if (G[j].pixel >= 0 && G[j].alive) take_direction(s, &G[j], into_lobe(&G[j], wl));
        } else if (reuse_now && cat == CAT_HYBRID && (p->opts & ORC_OPT_HYBRID_DONOR)) {
            /* hybrid group, donor reading (an option, not the paper's rule): the
             * diffuse members reuse the first diffuse member's own cosine sample,
             * the glossy/specular members keep theirs; every direction keeps its
             * sampling density, so the estimate stays unbiased */
            int donor = -1;
            for (uint32_t j = 0; j < K && donor < 0; ++j)
                if (G[j].pixel >= 0 && G[j].alive && G[j].cls == CLS_DIFFUSE) donor = (int)j;
            f3 wl = G[donor].wl;
            for (uint32_t j = 0; j < K; ++j)
                if (G[j].pixel >= 0 && G[j].alive && G[j].cls == CLS_DIFFUSE)
                    take_direction(s, &G[j], into_lobe(&G[j], wl));
        } else if (reuse_now && cat == CAT_HYBRID) {
            /* hybrid group: diffuse members take the normalised tangent-space sum of
             * the valid glossy/specular exit directions */
            for (uint32_t j = 0; j < K; ++j) {
                int use = G[j].pixel >= 0 && G[j].alive && G[j].cls == CLS_GLOSSY && G[j].valid;
                sumbuf[j] = use ? G[j].wl : f3m(0.0f, 0.0f, 0.0f);
            }
            f3 v = tree_sum(sumbuf, K);
            float l2 = f3dot(v, v);
            f3 wl;
            int keep_rough = 0;
            if (l2 > 0.0f) {
                float l = sqrtf(l2);
                wl = f3m(v.x / l, v.y / l, v.z / l);
                /* a rough GGX member (roughness threshold) keeps its own cosine
                 * sample: its weight pi f at the glossy average, near its own
                 * specular peak, would be far above 1 */
                keep_rough = 1;
            } else {
                /* no valid glossy sample: fall back to the diffuse-group rule
                 * among the diffuse members */
                int donor = -1;
                for (uint32_t j = 0; j < K && donor < 0; ++j)
                    if (G[j].pixel >= 0 && G[j].alive && G[j].cls == CLS_DIFFUSE) donor = (int)j;
                wl = G[donor].wl;
            }
            for (uint32_t j = 0; j < K; ++j)
                if (G[j].pixel >= 0 && G[j].alive && G[j].cls == CLS_DIFFUSE &&
                    !(keep_rough && G[j].cosgl))
                    take_direction(s, &G[j], into_lobe(&G[j], wl));
        }
        /* glossy groups and the independent mode keep every member's own sample */
        for (uint32_t j = 0; j < K; ++j) {
            pstate* ps = &G[j];
            if (ps->pixel < 0) continue;
            uint32_t di = dbg_row + (uint32_t)ps->pixel;
            if (out->dbg_cat) {
                out->dbg_cat[di] = (uint8_t)cat;
                out->dbg_cls[di] = (uint8_t)(!ps->alive ? CLS_NONE
                                             : (ps->hemi < 0.0f ? DBG_CLS_TRANSLUCENT : ps->cls));
                out->dbg_flags[di] = (uint8_t)((ps->alive ? 1 : 0) | (ps->alive && ps->valid ? 2 : 0) |
                                               (ps->taint ? 4 : 0));
                f3 wv = ps->alive ? to_world(ps, ps->wl) : f3m(0.0f, 0.0f, 0.0f);
                f3 lv = ps->alive ? ps->wl : f3m(0.0f, 0.0f, 0.0f);
                out->dbg_local[3 * di + 0] = lv.x;
                out->dbg_local[3 * di + 1] = lv.y;
                out->dbg_local[3 * di + 2] = lv.z;
                out->dbg_world[3 * di + 0] = wv.x;
                out->dbg_world[3 * di + 1] = wv.y;
                out->dbg_world[3 * di + 2] = wv.z;
            }
            if (!ps->alive) continue;
            if (!ps->valid) {
                ps->alive = 0;
                continue;
            }
            double o2[3];
            spawn_point(ps, ps->wl.z < 0.0f ? -1.0 : 1.0, o2);
            for (int k = 0; k < 3; ++k) ps->o[k] = o2[k];
            ps->d = to_world(ps, ps->wl);
            ps->pdf = bsdf_pdf(s, ps, ps->wl);
            for (int k = 0; k < 3; ++k) ps->beta[k] = ps->beta[k] * ps->w[k];
        }
    }
}

/* After the last secondary ray of a path only the environment (miss) or an emitter's
 * radiance where that ray ended is added. */
static void final_step(const orc_scene* s, const orc_params* p, pstate* slot, uint32_t m) {
    /* after the last secondary ray only the environment or an emitter is added */
    for (uint32_t j = 0; j < m; ++j) {
        pstate* ps = &slot[j];
        if (ps->pixel < 0) continue;
        if (ps->alive) {
            if (ps->hit < 0) {
                for (int k = 0; k < 3; ++k) ps->L[k] += (double)(ps->beta[k] * s->env[k]);
            } else if (s->mat_type[s->tri_mat[ps->hit]] == MAT_EMITTER) {
                const float* mp = &s->mat_params[7 * s->tri_mat[ps->hit]];
                double wb = (p->opts & ORC_OPT_NEE) ? emit_weight(s, ps) : 1.0;
                for (int k = 0; k < 3; ++k) ps->L[k] += (double)(ps->beta[k] * mp[4 + k]) * wb;
            }
        }
    }
}

void orc_render_tiles(const orc_scene* s, const orc_camera* cam, const orc_params* p, uint32_t tile_begin,
                      uint32_t tile_end, orc_outputs* out) {
    const uint32_t W = p->tile_w, H = p->tile_h, m = W * H, K = p->k;
    const uint32_t w = cam->width, h = cam->height, npx = w * h;
    const uint32_t ntx = (w + W - 1) / W;
    const uint32_t B = p->max_bounces;
    cam_basis cb = make_camera(cam);
    uint32_t* sigma = (uint32_t*)malloc(sizeof(uint32_t) * m);
    pstate* slot = (pstate*)malloc(sizeof(pstate) * m);
    f3* sumbuf = (f3*)malloc(sizeof(f3) * K);
    uint64_t cnt_local[5] = {0, 0, 0, 0, 0};

    for (uint32_t si = 0; si < p->spp; ++si) {
        const uint32_t f = p->frame_base + si;
        for (uint32_t tile = tile_begin; tile < tile_end; ++tile) {
            const uint32_t tx = tile % ntx, ty = tile / ntx;
            /* Sec. 3.3: shuffle the tile's pixel numbers; the slot of pixel i is sigma[i] */
            orc_tile_sigma(W, H, tile, f, p->seed, (int)p->interleave, sigma, NULL);
            for (uint32_t j = 0; j < m; ++j) slot[j].pixel = -1;
            for (uint32_t i = 0; i < m; ++i) {
                uint32_t px = tx * W + i % W, py = ty * H + i / W;
                pstate* ps = &slot[sigma[i]];
                if (px >= w || py >= h) continue; /* partial tile at the image border */
                ps->pixel = (int32_t)(py * w + px);
                ps->alive = 1;
                ps->taint = 0;
                ps->staint = 0;
                ps->pdf = 0.0;
                ps->beta[0] = ps->beta[1] = ps->beta[2] = 1.0f;
                ps->L[0] = ps->L[1] = ps->L[2] = 0.0;
                uint32_t hc[4];
                philox_seed(p->seed, (uint32_t)ps->pixel, f, 0, TAG_CAMERA, hc);
                ps->d = camera_dir(&cb, w, h, px, py, to_unit(hc[0]), to_unit(hc[1]));
                ps->o[0] = cb.pos.x;
                ps->o[1] = cb.pos.y;
                ps->o[2] = cb.pos.z;
                ps->hit = -1;
                capture_ray(ps, out, (uint32_t)ps->pixel);
                trace_path(s, ps, cnt_local);
                cnt_local[0]++;
                if (out->dbg_prim) out->dbg_prim[ps->pixel] = ps->hit;
                if (out->dbg_t) out->dbg_t[ps->pixel] = (float)ps->t;
            }
            for (uint32_t b = 1; b <= B; ++b) {
                shade_step(s, p, f, b, m, slot, sumbuf, out, (b - 1) * npx, cnt_local);
                /* trace the secondary rays of bounce b */
                for (uint32_t j = 0; j < m; ++j) {
                    pstate* ps = &slot[j];
                    if (ps->pixel < 0 || !ps->alive) continue;
                    capture_ray(ps, out, b * npx + (uint32_t)ps->pixel);
                    trace_path(s, ps, cnt_local);
                    cnt_local[1]++;
                    if (out->dbg_prim) out->dbg_prim[b * npx + (uint32_t)ps->pixel] = ps->hit;
                    if (out->dbg_t) out->dbg_t[b * npx + (uint32_t)ps->pixel] = (float)ps->t;
                }
            }
            final_step(s, p, slot, m);
            for (uint32_t j = 0; j < m; ++j) {
                pstate* ps = &slot[j];
                if (ps->pixel < 0) continue;
                for (int k = 0; k < 3; ++k) out->accum[3 * ps->pixel + k] += ps->L[k];
                if (out->taint && (ps->taint || ps->staint)) out->taint[ps->pixel] = 1;
            }
        }
    }
    if (out->counters)
        for (int k = 0; k < 5; ++k) out->counters[k] += cnt_local[k];
    free(sigma);
    free(slot);
    free(sumbuf);
}

/* Replay of one shading step on another renderer's captured state (see oracle.h): the tile's
 * slots are filled from the inputs of trace b-1 (ray, hit, throughput), then the same
 * shade_step (b <= B) or final_step (b = B + 1) as orc_render_tiles runs on them, so every
 * stage after the trace is recomputed from exactly the state the other renderer had. */
void orc_replay_step(const orc_scene* s, const orc_camera* cam, const orc_params* p, uint32_t frame, uint32_t bounce,
                     uint32_t tile_begin, uint32_t tile_end, const orc_replay_in* in, orc_replay_out* out) {
    const uint32_t W = p->tile_w, H = p->tile_h, m = W * H, K = p->k;
    const uint32_t w = cam->width, h = cam->height;
    const uint32_t ntx = (w + W - 1) / W;
    uint32_t* sigma = (uint32_t*)malloc(sizeof(uint32_t) * m);
    pstate* slot = (pstate*)malloc(sizeof(pstate) * m);
    f3* sumbuf = (f3*)malloc(sizeof(f3) * K);
    uint64_t cnt[5] = {0, 0, 0, 0, 0};
    orc_outputs dbg;
    memset(&dbg, 0, sizeof(dbg));
    dbg.dbg_cat = out->cat;
    dbg.dbg_cls = out->cls;
    dbg.dbg_flags = out->flags;
    dbg.dbg_local = out->local;
    dbg.dbg_world = out->world;
    for (uint32_t tile = tile_begin; tile < tile_end; ++tile) {
        const uint32_t tx = tile % ntx, ty = tile / ntx;
        orc_tile_sigma(W, H, tile, frame, p->seed, (int)p->interleave, sigma, NULL);
        for (uint32_t j = 0; j < m; ++j) slot[j].pixel = -1;
        for (uint32_t i = 0; i < m; ++i) {
            uint32_t px = tx * W + i % W, py = ty * H + i / W;
            if (px >= w || py >= h) continue;
            pstate* ps = &slot[sigma[i]];
            const uint32_t pix = py * w + px;
            memset(ps, 0, sizeof(*ps));
            ps->pixel = (int32_t)pix;
            ps->alive = in->prim[pix] != -2; /* -2: the path ended before trace b-1 */
            ps->hit = in->prim[pix];
            ps->t = (double)in->t[pix];
            for (int k = 0; k < 3; ++k) {
                ps->o[k] = (double)in->ray[8 * pix + k];
                ps->beta[k] = in->beta[4 * pix + k];
            }
            ps->d = f3m(in->ray[8 * pix + 4], in->ray[8 * pix + 5], in->ray[8 * pix + 6]);
            ps->pdf = (double)in->beta[4 * pix + 3];
            ps->hemi = 1.0f;
        }
        if (bounce <= p->max_bounces) {
            shade_step(s, p, frame, bounce, m, slot, sumbuf, &dbg, 0, cnt);
        } else {
            final_step(s, p, slot, m);
        }
        for (uint32_t j = 0; j < m; ++j) {
            const pstate* ps = &slot[j];
            if (ps->pixel < 0) continue;
            const uint32_t pix = (uint32_t)ps->pixel;
            const int cont = bounce <= p->max_bounces && ps->alive;
            for (int k = 0; k < 3; ++k) {
                if (out->dL) out->dL[3 * pix + k] = ps->L[k];
                if (out->next_o) out->next_o[3 * pix + k] = cont ? ps->o[k] : NAN;
                if (out->next_beta) out->next_beta[3 * pix + k] = cont ? ps->beta[k] : NAN;
            }
            if (out->next_pdf) out->next_pdf[pix] = cont ? ps->pdf : NAN;
            if (out->next_alive) out->next_alive[pix] = (uint8_t)cont;
            if (out->staint) out->staint[pix] = (uint8_t)ps->staint;
        }
    }
    free(sigma);
    free(slot);
    free(sumbuf);
}
