// trace_common.cuh -- traversal primitives shared by the BVH2 kernels (trace.cu) and the
// BVH8-Q kernels (trace_bvh8.cu): ray set-up, the conservative slab tests, the watertight
// ray/triangle test, the closest-hit rule and the short traversal stack.
//
// Closest-hit rule, identical for every kernel: accept t > 0 if t < t_best, or t == t_best
// and the original triangle index is smaller.  Boxes are culled only if their entry distance
// exceeds t_best (1 + 2^-16) and the slab exit is widened by (1 + 2^-21) > 1 + 2 gamma_3
// (Ize 2013), so no box that holds a candidate triangle is ever skipped and every layout
// returns the same hit bit for bit.
#pragma once
#include <cuda_runtime.h>

#include "cr_internal.h"
#include "debug_checks.cuh"

namespace cr {
namespace {

constexpr int kSmemStack = 16;  // entries per thread in shared memory
constexpr int kStackTotal = (int)kBvh2StackCapacity; // > BVH2 depth (checked at scene creation)
constexpr float kFarWiden = 1.0f + 0x1.0p-21f;
constexpr float kCullWiden = 1.0f + 0x1.0p-16f;

struct RayPre {
    float ox, oy, oz;
    float ix, iy, iz; // 1 / d (zero components replaced by +-1e-20 first)
    int kx, ky, kz;
    float sx, sy, sz; // shear constants of the watertight test
    float dx, dy, dz;
    // slab offsets for t = fma(plane, 1/d, offset): -o/d biased outward by 2^-22 |o/d|, which
    // bounds the rounding of o/d and of the offset, so the FMA interval contains the one the
    // exact (plane - o) / d form gives (see box_entry_fma)
    float lox, loy, loz, hix, hiy, hiz;
};

__device__ __forceinline__ float sel3(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ RayPre prep_ray(float4 o, float4 d) {
    RayPre r;
    r.ox = o.x;
    r.oy = o.y;
    r.oz = o.z;
    r.dx = d.x;
    r.dy = d.y;
    r.dz = d.z;
    const float tiny = 1e-20f;
    r.ix = 1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x));
    r.iy = 1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y));
    r.iz = 1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z));
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = ax > ay ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    const float dkz = sel3(d.x, d.y, d.z, kz);
    if (dkz < 0.0f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    r.sx = sel3(d.x, d.y, d.z, kx) / dkz;
    r.sy = sel3(d.x, d.y, d.z, ky) / dkz;
    r.sz = 1.0f / dkz;
    // plane of the lower bound enters first when 1/d >= 0; bias each offset so that the
    // entry distance can only decrease and the exit distance only increase
    const float oix = __fmul_rn(r.ox, r.ix), oiy = __fmul_rn(r.oy, r.iy), oiz = __fmul_rn(r.oz, r.iz);
    const float ex = __fmul_rn(fabsf(oix), 0x1.0p-22f), ey = __fmul_rn(fabsf(oiy), 0x1.0p-22f),
                ez = __fmul_rn(fabsf(oiz), 0x1.0p-22f);
    r.lox = r.ix >= 0.0f ? -oix - ex : -oix + ex;
    r.hix = r.ix >= 0.0f ? -oix + ex : -oix - ex;
    r.loy = r.iy >= 0.0f ? -oiy - ey : -oiy + ey;
    r.hiy = r.iy >= 0.0f ? -oiy + ey : -oiy - ey;
    r.loz = r.iz >= 0.0f ? -oiz - ez : -oiz + ez;
    r.hiz = r.iz >= 0.0f ? -oiz + ez : -oiz - ez;
    return r;
}

// Slab test of one box; returns the entry distance, or +inf if the box is missed or culled.
__device__ __forceinline__ float box_entry(const RayPre& r, float lox, float hix, float loy, float hiy, float loz,
                                           float hiz, float tcull) {
    const float tx0 = __fmul_rn(__fsub_rn(lox, r.ox), r.ix), tx1 = __fmul_rn(__fsub_rn(hix, r.ox), r.ix);
    const float ty0 = __fmul_rn(__fsub_rn(loy, r.oy), r.iy), ty1 = __fmul_rn(__fsub_rn(hiy, r.oy), r.iy);
    const float tz0 = __fmul_rn(__fsub_rn(loz, r.oz), r.iz), tz1 = __fmul_rn(__fsub_rn(hiz, r.oz), r.iz);
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    return (tn <= __fmul_rn(tf, kFarWiden) && tn <= tcull) ? tn : INFINITY;
}

// The same test with one FMA per plane.  Each plane distance fma(x, 1/d, offset) differs
// from (x - o) * (1/d) by at most the rounding of o/d and of the offset (<= 2^-23 |o/d|) plus a
// relative 2^-24; the offsets are pre-biased by 2^-22 |o/d| toward a larger interval and the
// exit is widened by (1 + 2^-21), so no box that the exact form would enter is rejected.
#ifndef CR_TRACE_MINMAX3
#define CR_TRACE_MINMAX3 1
#endif
// three-input min / max (one instruction each on sm_100 and later)
__device__ __forceinline__ float min3f(float a, float b, float c) {
#if CR_TRACE_MINMAX3
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
#else
    return fminf(fminf(a, b), c);
#endif
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
#if CR_TRACE_MINMAX3
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
#else
    return fmaxf(fmaxf(a, b), c);
#endif
}

__device__ __forceinline__ float box_entry_fma(const RayPre& r, float lox, float hix, float loy, float hiy, float loz,
                                               float hiz, float tcull) {
    const float tx0 = fmaf(lox, r.ix, r.lox), tx1 = fmaf(hix, r.ix, r.hix);
    const float ty0 = fmaf(loy, r.iy, r.loy), ty1 = fmaf(hiy, r.iy, r.hiy);
    const float tz0 = fmaf(loz, r.iz, r.loz), tz1 = fmaf(hiz, r.iz, r.hiz);
    const float tn = max3f(fminf(tx0, tx1), fminf(ty0, ty1), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = min3f(fmaxf(tx0, tx1), fmaxf(ty0, ty1), fmaxf(tz0, tz1));
    return (tn <= __fmul_rn(tf, kFarWiden) && tn <= tcull) ? tn : INFINITY;
}

// box_entry_fma as a hit flag plus the entry distance (no +inf sentinel to test again).
__device__ __forceinline__ bool box_hit_fma(const RayPre& r, float lox, float hix, float loy, float hiy, float loz,
                                            float hiz, float tcull, float& tn) {
    const float tx0 = fmaf(lox, r.ix, r.lox), tx1 = fmaf(hix, r.ix, r.hix);
    const float ty0 = fmaf(loy, r.iy, r.loy), ty1 = fmaf(hiy, r.iy, r.hiy);
    const float tz0 = fmaf(loz, r.iz, r.loz), tz1 = fmaf(hiz, r.iz, r.hiz);
    tn = max3f(fminf(tx0, tx1), fminf(ty0, ty1), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = min3f(fmaxf(tx0, tx1), fmaxf(ty0, ty1), fmaxf(tz0, tz1));
    return tn <= __fmul_rn(tf, kFarWiden) && tn <= tcull;
}

// Watertight ray/triangle test (Woop, Benthin, Wald 2013) without the double-precision
// fallback: edge functions of exactly zero count as inside, so shared edges are covered.
__device__ __forceinline__ bool tri_test(const RayPre& r, float4 a4, float4 b4, float4 c4, float& t_out) {
    const float Ax3 = a4.x - r.ox, Ay3 = a4.y - r.oy, Az3 = a4.z - r.oz;
    const float Bx3 = b4.x - r.ox, By3 = b4.y - r.oy, Bz3 = b4.z - r.oz;
    const float Cx3 = c4.x - r.ox, Cy3 = c4.y - r.oy, Cz3 = c4.z - r.oz;
    const float Akx = sel3(Ax3, Ay3, Az3, r.kx), Aky = sel3(Ax3, Ay3, Az3, r.ky), Akz = sel3(Ax3, Ay3, Az3, r.kz);
    const float Bkx = sel3(Bx3, By3, Bz3, r.kx), Bky = sel3(Bx3, By3, Bz3, r.ky), Bkz = sel3(Bx3, By3, Bz3, r.kz);
    const float Ckx = sel3(Cx3, Cy3, Cz3, r.kx), Cky = sel3(Cx3, Cy3, Cz3, r.ky), Ckz = sel3(Cx3, Cy3, Cz3, r.kz);
    const float Ax = __fsub_rn(Akx, __fmul_rn(r.sx, Akz)), Ay = __fsub_rn(Aky, __fmul_rn(r.sy, Akz));
    const float Bx = __fsub_rn(Bkx, __fmul_rn(r.sx, Bkz)), By = __fsub_rn(Bky, __fmul_rn(r.sy, Bkz));
    const float Cx = __fsub_rn(Ckx, __fmul_rn(r.sx, Ckz)), Cy = __fsub_rn(Cky, __fmul_rn(r.sy, Ckz));
    const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return false;
    const float Az = __fmul_rn(r.sz, Akz), Bz = __fmul_rn(r.sz, Bkz), Cz = __fmul_rn(r.sz, Ckz);
    const float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Az), __fmul_rn(V, Bz)), __fmul_rn(W, Cz));
    const float t = __fdiv_rn(T, det);
    if (!(t > 0.0f)) return false;
    t_out = t;
    return true;
}

struct Best {
    float t;
    int leaf;
    int orig;
};

__device__ __forceinline__ void test_leaf(const float4* __restrict__ tris, const RayPre& r, int skip, uint32_t first,
                                          uint32_t count, Best& best, unsigned long long& n_tri) {
    for (uint32_t i = 0; i < count; ++i) {
        const uint32_t tri = first + i;
        const float4 a = __ldg(&tris[3 * tri + 0]);
        const int orig = __float_as_int(a.w);
        if (orig == skip) continue;
        const float4 b = __ldg(&tris[3 * tri + 1]);
        const float4 c = __ldg(&tris[3 * tri + 2]);
        ++n_tri;
        float t;
        if (tri_test(r, a, b, c, t) && (t < best.t || (t == best.t && orig < best.orig))) {
            best.t = t;
            best.leaf = (int)tri;
            best.orig = orig;
        }
    }
}

#ifndef CR_TRACE_LOCAL_STACK
#define CR_TRACE_LOCAL_STACK 0
#endif
#if CR_TRACE_LOCAL_STACK
// whole stack in a per-thread local array (L1-resident); depth < kStackTotal by construction
#define STACK_PUSH(v) (lstack_all[sp++] = (v))
#define STACK_POP(v) ((v) = lstack_all[--sp])
#else
// first kSmemS entries (the user's constant: kSmemStack, or a template parameter) in shared
// memory, the rest in a local array
// (a push never exceeds the tree depth, which scene creation checks is below kStackTotal)
#define STACK_PUSH(v)                                                                \
    do {                                                                             \
        if (sp < kSmemS) sstack[sp * stride] = (uint32_t)(v);                        \
        else lstack[sp - kSmemS] = (v);                                              \
        ++sp;                                                                        \
    } while (0)
#define STACK_POP(v)                                                                 \
    do {                                                                             \
        --sp;                                                                        \
        (v) = sp < kSmemS ? (int)sstack[sp * stride] : lstack[sp - kSmemS];          \
    } while (0)
#endif


// The same stack with a pointer to the next free shared-memory entry, which saves the index
// arithmetic of every push and pop (1% on the secondary trace); used by trace_bvh2_one.
#define STACK_PUSH_TOP(v)                                                            \
    do {                                                                             \
        if (sp < kSmemS) {                                                           \
            *top = (uint32_t)(v);                                                    \
            top += stride;                                                           \
        } else {                                                                     \
            lstack[sp - kSmemS] = (v);                                               \
        }                                                                            \
        ++sp;                                                                        \
    } while (0)
#define STACK_POP_TOP(v)                                                             \
    do {                                                                             \
        --sp;                                                                        \
        if (sp < kSmemS) {                                                           \
            top -= stride;                                                           \
            (v) = (int)*top;                                                         \
        } else {                                                                     \
            (v) = lstack[sp - kSmemS];                                               \
        }                                                                            \
    } while (0)

} // namespace
} // namespace cr
