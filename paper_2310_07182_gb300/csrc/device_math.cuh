// device_math.cuh -- device arithmetic of the path tracer: counter-based RNG, FP32
// operations with a fixed rounding sequence, sine/cosine polynomial, BSDF samplers and the
// tangent frame.
//
// Every floating-point step that feeds a ray direction uses the explicit round-to-nearest
// intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn): the compiler may not fuse
// them into FMAs, so a direction is the same bit pattern on every run and launch shape.
#pragma once
#include <cstdint>

namespace cr {
namespace dev {

// Counter tags (counter = (pixel or tile, frame, bounce or tag, tag)).
constexpr uint32_t kTagCamera = 0x43414D45u;     // "CAME"
constexpr uint32_t kTagBsdf = 0x42534446u;       // "BSDF"
constexpr uint32_t kTagInterleave = 0x494E544Cu; // "INTL"
constexpr uint32_t kTagLight = 0x4C495445u;      // "LITE"

constexpr uint32_t kMatLambert = 0, kMatGGX = 1, kMatMirror = 2, kMatEmitter = 3, kMatDielectric = 4,
                   kMatTranslucent = 5;
constexpr int kClsNone = 0, kClsDiffuse = 1, kClsGlossy = 2;
constexpr int kCatEmpty = 0, kCatDiffuse = 1, kCatGlossy = 2, kCatHybrid = 3;

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds; each round multiplies words 0 and 2 by
// the round multipliers, swaps in the high halves xor'ed with the other words and the
// round key, and the key is bumped by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint32_t k0, uint32_t k1, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
__device__ __forceinline__ uint4 philox_seed(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
    return philox((uint32_t)seed, (uint32_t)(seed >> 32), make_uint4(c0, c1, c2, c3));
}
// Upper 24 bits as a float in [0, 1) (exact).
__device__ __forceinline__ float unit24(uint32_t x) { return __fmul_rn(__uint2float_rn(x >> 8), 0x1.0p-24f); }

// FP32 operations in a fixed order.
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fq(float a) { return __fsqrt_rn(a); }

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ float dot3(V3 a, V3 b) { return fa(fa(fm(a.x, b.x), fm(a.y, b.y)), fm(a.z, b.z)); }
__device__ __forceinline__ V3 sub3(V3 a, V3 b) { return v3(fs(a.x, b.x), fs(a.y, b.y), fs(a.z, b.z)); }
__device__ __forceinline__ V3 cross3(V3 a, V3 b) {
    return v3(fs(fm(a.y, b.z), fm(a.z, b.y)), fs(fm(a.z, b.x), fm(a.x, b.z)), fs(fm(a.x, b.y), fm(a.y, b.x)));
}
__device__ __forceinline__ V3 normalize3(V3 a) {
    const float l = fq(dot3(a, a));
    if (l == 0.0f) return v3(0.0f, 0.0f, 1.0f);
    return v3(fd(a.x, l), fd(a.y, l), fd(a.z, l));
}

// sin and cos for |x| <= pi/4: Taylor polynomials of degree 11 and 12 (coefficients 1/n!
// rounded to float), Horner's rule.
__device__ __forceinline__ void sincos_poly(float x, float& s, float& c) {
    const float x2 = fm(x, x);
    float ps = -0x1.ae6456p-26f;
    ps = fa(fm(ps, x2), 0x1.71de3ap-19f);
    ps = fa(fm(ps, x2), -0x1.a01a02p-13f);
    ps = fa(fm(ps, x2), 0x1.111112p-7f);
    ps = fa(fm(ps, x2), -0x1.555556p-3f);
    s = fa(x, fm(fm(x, x2), ps));
    float pc = 0x1.1eed8ep-29f;
    pc = fa(fm(pc, x2), -0x1.27e4fcp-22f);
    pc = fa(fm(pc, x2), 0x1.a01a02p-16f);
    pc = fa(fm(pc, x2), -0x1.6c16c2p-10f);
    pc = fa(fm(pc, x2), 0x1.555556p-5f);
    pc = fa(fm(pc, x2), -0x1.0p-1f);
    c = fa(1.0f, fm(x2, pc));
}

constexpr float kPi4 = 0x1.921fb6p-1f;
constexpr float kPi2 = 0x1.921fb6p+0f;
constexpr float kInvSqrt2 = 0x1.6a09e6p-1f;

// Cosine-weighted hemisphere direction from the concentric square-to-disk map of Shirley
// and Chiu (1997); in the wedge |a| <= |b| the angle pi/2 - (pi/4)(a/b) is taken through
// sin/cos swapped so the polynomial argument stays within [-pi/4, pi/4].
__device__ __forceinline__ V3 sample_cosine(float u1, float u2) {
    const float a = fs(fm(2.0f, u1), 1.0f);
    const float b = fs(fm(2.0f, u2), 1.0f);
    float x, y;
    if (a == 0.0f && b == 0.0f) {
        x = 0.0f;
        y = 0.0f;
    } else if (fabsf(a) > fabsf(b)) {
        float s, c;
        sincos_poly(fm(kPi4, fd(b, a)), s, c);
        x = fm(a, c);
        y = fm(a, s);
    } else {
        float s, c;
        sincos_poly(fm(kPi4, fd(a, b)), s, c);
        x = fm(b, s);
        y = fm(b, c);
    }
    const float zz = fs(fs(1.0f, fm(x, x)), fm(y, y));
    return v3(x, y, fq(zz > 0.0f ? zz : 0.0f));
}

// cos/sin of 2 pi u: quadrant q = floor(4u) and a residual angle psi in [-pi/4, pi/4)
// about the quadrant's centre; rotation by pi/4 + q pi/2 is exact except the 1/sqrt2.
__device__ __forceinline__ void sincos_2pi(float u, float& cphi, float& sphi) {
    const float t = fm(4.0f, u);
    int q = (int)t;
    q = q > 3 ? 3 : q;
    const float fr = fs(t, (float)q);
    float s, c;
    sincos_poly(fm(fs(fr, 0.5f), kPi2), s, c);
    const float c0 = fm(fs(c, s), kInvSqrt2);
    const float s0 = fm(fa(c, s), kInvSqrt2);
    if (q == 0) { cphi = c0; sphi = s0; }
    else if (q == 1) { cphi = -s0; sphi = c0; }
    else if (q == 2) { cphi = -c0; sphi = -s0; }
    else { cphi = s0; sphi = -c0; }
}

__device__ __forceinline__ float smith_g1(float vz, float a2) {
    const float z2 = fm(vz, vz);
    float t2 = fd(fs(1.0f, z2), z2);
    t2 = t2 < 0.0f ? 0.0f : t2;
    return fd(2.0f, fa(1.0f, fq(fa(1.0f, fm(a2, t2)))));
}

// GGX reflection (Walter et al. 2007): the microfacet normal m is drawn from D(m)(m.n)
// and wo is reflected about it.  The weight f cos / pdf equals F G (wo.m) / (wo.z m.z)
// with Schlick's F (F0 = albedo) and Smith's separable G = G1(wo) G1(wi).
__device__ __forceinline__ bool sample_ggx(V3 wo, float alpha, const float* f0, float u1, float u2, V3& wi,
                                           float* w) {
    const float a2 = fm(alpha, alpha);
    const float tan2 = fd(fm(a2, u1), fs(1.0f, u1));
    const float ct = fd(1.0f, fq(fa(1.0f, tan2)));
    const float st2 = fs(1.0f, fm(ct, ct));
    const float st = fq(st2 > 0.0f ? st2 : 0.0f);
    float cphi, sphi;
    sincos_2pi(u2, cphi, sphi);
    const V3 m = v3(fm(st, cphi), fm(st, sphi), ct);
    const float d = dot3(wo, m);
    const float d2 = fm(2.0f, d);
    wi = v3(fs(fm(d2, m.x), wo.x), fs(fm(d2, m.y), wo.y), fs(fm(d2, m.z), wo.z));
    if (!(wo.z > 0.0f) || !(d > 0.0f) || !(wi.z > 0.0f)) {
        w[0] = w[1] = w[2] = 0.0f;
        return false;
    }
    const float g = fm(smith_g1(wo.z, a2), smith_g1(wi.z, a2));
    const float om = fs(1.0f, d);
    const float om2 = fm(om, om);
    const float p5 = fm(fm(om2, om2), om);
    const float den = fm(wo.z, m.z);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float F = fa(f0[k], fm(fs(1.0f, f0[k]), p5));
        w[k] = fd(fm(fm(F, g), d), den);
    }
    return true;
}

// Smooth dielectric (IOR eta inside, 1 outside; the inside lies behind the triangle's front
// face): unpolarised Fresnel reflectance F from e = eta_i / eta_t, reflection when u < F
// (always under total internal reflection, sin^2 t >= 1), else Snell refraction
// wi = (-e wo.x, -e wo.y, -cos t).  The weight is the tint for both branches.
__device__ __forceinline__ V3 sample_dielectric(V3 wo, float eta, bool front, float u) {
    const float eta_i = front ? 1.0f : eta, eta_t = front ? eta : 1.0f;
    const float e = fd(eta_i, eta_t);
    const float ci = wo.z;
    const float s2 = fm(fm(e, e), fs(1.0f, fm(ci, ci)));
    float F = 1.0f, ct = 0.0f;
    if (s2 < 1.0f) {
        ct = fq(fs(1.0f, s2));
        const float rs = fd(fs(fm(eta_i, ci), fm(eta_t, ct)), fa(fm(eta_i, ci), fm(eta_t, ct)));
        const float rp = fd(fs(fm(eta_t, ci), fm(eta_i, ct)), fa(fm(eta_t, ci), fm(eta_i, ct)));
        F = fm(0.5f, fa(fm(rs, rs), fm(rp, rp)));
    }
    if (u < F) return v3(-wo.x, -wo.y, wo.z);
    return v3(-fm(e, wo.x), -fm(e, wo.y), -ct);
}

// GGX reflection value f(wo, wi) in the tangent frame: the density sample_ggx draws from,
// D(h) G1(wo) G1(wi) F(wo.h) / (4 wo.z wi.z) with h = normalize(wo + wi) and
// D(h) = alpha^2 / (pi (1 + (alpha^2 - 1) h.z^2)^2) (Walter et al. 2007); 0 below either side.
__device__ __forceinline__ void eval_ggx(V3 wo, V3 wi, float alpha, const float* f0, float* f) {
    f[0] = f[1] = f[2] = 0.0f;
    if (!(wo.z > 0.0f) || !(wi.z > 0.0f)) return;
    const V3 hs = v3(fa(wo.x, wi.x), fa(wo.y, wi.y), fa(wo.z, wi.z));
    const float hl2 = dot3(hs, hs);
    if (!(hl2 > 0.0f)) return;
    const float hl = fq(hl2);
    const V3 h = v3(fd(hs.x, hl), fd(hs.y, hl), fd(hs.z, hl));
    const float oh = dot3(wo, h);
    if (!(oh > 0.0f)) return;
    const float a2 = fm(alpha, alpha);
    const float q = fa(1.0f, fm(fs(a2, 1.0f), fm(h.z, h.z)));
    const float D = fd(a2, fm(3.14159265358979f, fm(q, q)));
    const float g = fm(smith_g1(wo.z, a2), smith_g1(wi.z, a2));
    const float om = fs(1.0f, oh);
    const float om2 = fm(om, om);
    const float p5 = fm(fm(om2, om2), om);
    const float den = fm(4.0f, fm(wo.z, wi.z));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float F = fa(f0[k], fm(fs(1.0f, f0[k]), p5));
        f[k] = fd(fm(fm(D, g), F), den);
    }
}

// Solid-angle density with which sample_ggx draws wi: D(h) h.z / (4 wo.h), h = normalize(wo + wi)
// (the microfacet normal has density D(h) h.z; reflection has Jacobian 1 / (4 wo.h)).
__device__ __forceinline__ float pdf_ggx(V3 wo, V3 wi, float alpha) {
    if (!(wo.z > 0.0f) || !(wi.z > 0.0f)) return 0.0f;
    const V3 hs = v3(fa(wo.x, wi.x), fa(wo.y, wi.y), fa(wo.z, wi.z));
    const float hl2 = dot3(hs, hs);
    if (!(hl2 > 0.0f)) return 0.0f;
    const float hl = fq(hl2);
    const V3 h = v3(fd(hs.x, hl), fd(hs.y, hl), fd(hs.z, hl));
    const float oh = dot3(wo, h);
    if (!(oh > 0.0f)) return 0.0f;
    const float a2 = fm(alpha, alpha);
    const float q = fa(1.0f, fm(fs(a2, 1.0f), fm(h.z, h.z)));
    const float D = fd(a2, fm(3.14159265358979f, fm(q, q)));
    return fd(fm(D, h.z), fm(4.0f, oh));
}

// Orthonormal basis (t, b, n) from a unit normal after Duff et al., "Building an
// Orthonormal Basis, Revisited" (JCGT 2017).  It depends on n only.
__device__ __forceinline__ void frame_from(V3 n, V3& t, V3& b) {
    const float sign = copysignf(1.0f, n.z);
    const float a = fd(-1.0f, fa(sign, n.z));
    const float bb = fm(fm(n.x, n.y), a);
    t = v3(fa(1.0f, fm(fm(fm(sign, n.x), n.x), a)), fm(sign, bb), -fm(sign, n.x));
    b = v3(bb, fa(sign, fm(fm(n.y, n.y), a)), -n.y);
}

__device__ __forceinline__ V3 local_to_world(V3 t, V3 b, V3 n, V3 l) {
    return v3(fa(fa(fm(t.x, l.x), fm(b.x, l.y)), fm(n.x, l.z)), fa(fa(fm(t.y, l.x), fm(b.y, l.y)), fm(n.y, l.z)),
              fa(fa(fm(t.z, l.x), fm(b.z, l.y)), fm(n.z, l.z)));
}

} // namespace dev
} // namespace cr
